// C ABI entry points (see include/lcp.h for the contract of each call).
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "index.cuh"
#include "sort.cuh"

namespace lcph {

static std::atomic<int64_t> g_launches{0};
static thread_local cudaError_t g_last_cuda = cudaSuccess;

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void note_use(lcp_index_s* x, cudaStream_t s) {
    for (int i = 0; i < x->nuses; ++i)
        if (x->uses[i].s == s) {
            cudaEventRecord(x->uses[i].e, s);
            return;
        }
    if (x->nuses == lcp_index_s::kMaxUses) {
        x->shared = true;  // too many streams to track
        return;
    }
    lcp_index_s::Use& u = x->uses[x->nuses];
    if (cudaEventCreateWithFlags(&u.e, cudaEventDisableTiming) != cudaSuccess) {
        x->shared = true;
        return;
    }
    u.s = s;
    cudaEventRecord(u.e, s);
    x->nuses++;
}

// One non-blocking stream per device for stream-ordered frees.
static cudaStream_t free_stream() {
    static cudaStream_t fs[64] = {nullptr};
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) return nullptr;
    if (!fs[dev]) cudaStreamCreateWithFlags(&fs[dev], cudaStreamNonBlocking);
    return fs[dev];
}

// ---- per-kernel event timing ----
struct KtRec {
    const char* name;
    cudaEvent_t a, b;
};
static std::atomic<bool> g_kt_on{false};
static std::atomic<bool> g_build_graph{true};  // lcp_build_graph
static std::mutex g_kt_mu;
static std::vector<KtRec> g_kt_pending;
static std::vector<cudaEvent_t> g_kt_pool;
static std::map<std::string, std::pair<double, int64_t>> g_kt_total;

static cudaEvent_t kt_event() {  // caller holds g_kt_mu
    cudaEvent_t e = nullptr;
    if (!g_kt_pool.empty()) {
        e = g_kt_pool.back();
        g_kt_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        e = nullptr;
    }
    return e;
}

static std::string g_kt_filter;  // time only kernels whose name starts with this ("" = all)

bool ktime_on() { return g_kt_on.load(std::memory_order_relaxed); }

void* ktime_begin(const char* name, cudaStream_t s) {
    {
        std::lock_guard<std::mutex> lk(g_kt_mu);
        if (!g_kt_filter.empty() && strncmp(name, g_kt_filter.c_str(), g_kt_filter.size()) != 0) return nullptr;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
    std::lock_guard<std::mutex> lk(g_kt_mu);
    KtRec* r = new (std::nothrow) KtRec{name, kt_event(), kt_event()};
    if (!r || !r->a || !r->b) {
        if (r) {
            if (r->a) g_kt_pool.push_back(r->a);
            if (r->b) g_kt_pool.push_back(r->b);
            delete r;
        }
        return nullptr;
    }
    cudaEventRecord(r->a, s);
    return r;
}

void ktime_end(void* token, cudaStream_t s) {
    KtRec* r = static_cast<KtRec*>(token);
    cudaEventRecord(r->b, s);
    std::lock_guard<std::mutex> lk(g_kt_mu);
    g_kt_pending.push_back(*r);
    delete r;
}

int cuda_status(cudaError_t e) {
    g_last_cuda = e;
    if (e == cudaErrorMemoryAllocation) return LCP_ERR_OOM;
    return LCP_ERR_CUDA;
}

// Library-wide device status word (one per device, allocated on first use).
static int* g_status[64] = {nullptr};
static std::mutex g_status_mu;

int* lib_status_word() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_status_mu);
    if (!g_status[dev]) {
        int* p = nullptr;
        if (cudaMalloc((void**)&p, sizeof(int)) != cudaSuccess) return nullptr;
        cudaMemset(p, 0, sizeof(int));
        g_status[dev] = p;
    }
    return g_status[dev];
}

// The same word if it exists already, else null (never allocates).
int* lib_status_word_if_any() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_status_mu);
    return g_status[dev];
}

int sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (!cache[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = n > 0 ? n : 148;
    }
    return cache[dev];
}

int scan_topk_device(const void* d_tokens, int64_t N, int tb, int L, const void* d_queries,
                     int64_t Q, int k, int32_t* d_out_ids, uint8_t* d_out_lcp, cudaStream_t s);

static int valid_fmt(const lcp_format_t& f) {
    return (f.token_bytes == 1 || f.token_bytes == 2) && f.L >= 1 && f.L <= LCP_MAX_L;
}

// An index may also hold rows of up to LCP_MAX_L_WIDE tokens when it is built
// for top-1 only (max_k = 1): lcp_top1_wide answers it with 16-bit LCPs.
static int valid_build_fmt(const lcp_format_t& f, int32_t max_k) {
    return valid_fmt(f) || ((f.token_bytes == 1 || f.token_bytes == 2) && f.L > LCP_MAX_L &&
                            f.L <= LCP_MAX_L_WIDE && max_k == 1);
}

// Index memory comes from the device's stream-ordered pool, which is told to
// keep freed memory (release threshold = max), so destroying and rebuilding
// indexes in a serving loop reuses memory instead of paying cudaMalloc/cudaFree.
static void retain_pool_memory() {
    static std::once_flag once[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::call_once(once[dev], [dev]() {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    });
}

// Frees with cudaFreeAsync on stream s (the build's own stream on failure) or,
// with s == nullptr and the device idle, synchronously.
static void free_index_memory(lcp_index_s* x, cudaStream_t s) {
    if (x->arena) {
        if (s) cudaFreeAsync(x->arena, s);
        else cudaFree(x->arena);
    }
    x->arena = nullptr;
    x->buf[0] = lcp_buffers();
    x->buf[1] = lcp_buffers();
}


constexpr int kTieListMinK = 16;

// ---- the build as one CUDA graph ----
//
// A build is some sixty launches; replayed as one graph they reach the
// device as a unit instead of one by one.  Each thread keeps, per device, a
// capture stream, the instantiated graph of its last build (updated in place
// for the next one: only pointers and grid sizes change) and the build's
// scratch block (grown when a larger build comes; reuse across streams waits
// on the event recorded after the graph that used it last).
struct GraphBuildState {
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    void* scratch = nullptr;
    size_t bytes = 0;
    cudaEvent_t scratch_free = nullptr;
    cudaEvent_t chk = nullptr;
    // What the instantiated graph was captured for: every pointer and size
    // it holds follows from these (the index's arrays are carved from its
    // arena by the format, capacity and K), so a build with the same
    // signature -- the pool usually hands a rebuilt index the same arena --
    // relaunches it without a new capture.  The host-side fields the
    // capture set on the index are kept with it.
    struct Sig {
        const void* tokens = nullptr;
        int64_t N = 0, cap = 0;
        void* arena = nullptr;
        void* scratch = nullptr;
        int tb = 0, L = 0, K = 0, max_k = 0;
        bool operator==(const Sig& o) const {
            return tokens == o.tokens && N == o.N && cap == o.cap && arena == o.arena && scratch == o.scratch &&
                   tb == o.tb && L == o.L && K == o.K && max_k == o.max_k;
        }
    } sig;
    bool sig_ok = false;
    int hlev = 0;
    int64_t hoff[lcpk::kMaxHLev + 1] = {0};
    int64_t hlen[lcpk::kMaxHLev + 1] = {0};
};

static GraphBuildState* graph_build_state() {
    static thread_local GraphBuildState st[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    GraphBuildState& g = st[dev];
    if (!g.cap && cudaStreamCreateWithFlags(&g.cap, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    if (!g.scratch_free && cudaEventCreateWithFlags(&g.scratch_free, cudaEventDisableTiming) != cudaSuccess)
        return nullptr;
    if (!g.chk && cudaEventCreateWithFlags(&g.chk, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    return &g;
}

// Launches the instantiated build graph on s, then waits for its mid-graph
// event and, when rows were left to the exact refinement, redoes the order.
static int launch_build_graph(GraphBuildState* g, lcp_index_s* x, const void* d_tokens, const lcpk::RowFmt& f,
                              int64_t N, cudaStream_t s, const uint32_t* huge) {
    LCP_CUDA_TRY(cudaStreamWaitEvent(s, g->scratch_free, 0));  // a graph on another stream used the scratch
    LCP_CUDA_TRY(cudaGraphLaunch(g->exec, s));
    LCP_CUDA_TRY(cudaEventRecord(g->scratch_free, s));
    LCP_CUDA_TRY(cudaEventSynchronize(g->chk));
    if (*huge != 0) {
        int rc = build_sorted_ids(d_tokens, f, N, x->buf[0].ids, x->status, s);
        if (rc == LCP_OK) rc = gather_rows_and_lcp(d_tokens, f, N, x->buf[0].ids, x->buf[0], x->W, s);
        if (rc == LCP_OK) rc = build_aux(x, s, false);
        if (rc != LCP_OK) return rc;
    }
    const cudaError_t le = cudaGetLastError();
    return le == cudaSuccess ? LCP_OK : cuda_status(le);
}

// Returns LCP_OK (built), LCP_PENDING (cannot run as a graph here; nothing
// was issued) or an error.  Rows in tie groups the on-device group sort does
// not take -- more than 2,048 rows sharing word 0, or a group of 33-2,048 in
// which a row shares word 1 with more than 64 others -- need the exact,
// host-driven refinement: their count lands in pinned memory behind an event
// recorded mid-graph, after the sort.  The host waits for that event (every
// build), then returns while the device runs the second half of the build;
// a nonzero count (rare: heavy duplication) redoes the order exactly on `s`.
static int graph_build(lcp_index_s* x, const void* d_tokens, int64_t N, cudaStream_t s) {
    GraphBuildState* g = graph_build_state();
    uint32_t* huge = pinned_words();
    if (!g || !huge) return LCP_PENDING;
    huge += 12;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return LCP_PENDING;
    const size_t need = build_scratch_bytes(N);
    if (g->bytes < need) {
        if (g->scratch) {
            LCP_CUDA_TRY(cudaStreamWaitEvent(s, g->scratch_free, 0));
            LCP_CUDA_TRY(cudaFreeAsync(g->scratch, s));
            g->scratch = nullptr;
            g->bytes = 0;
        }
        const size_t want = need + need / 4;
        LCP_CUDA_TRY(cudaMallocAsync(&g->scratch, want, s));
        g->bytes = want;
    }
    *huge = 0;
    lcpk::RowFmt f = lcpk::make_fmt(x->tb, x->L, d_tokens);
    GraphBuildState::Sig sig;
    sig.tokens = d_tokens;
    sig.N = N;
    sig.cap = x->cap;
    sig.arena = x->arena;
    sig.scratch = g->scratch;
    sig.tb = x->tb;
    sig.L = x->L;
    sig.K = x->K;
    sig.max_k = x->max_k;
    if (g->exec && g->sig_ok && sig == g->sig) {  // the same graph: relaunch it
        x->hlev = g->hlev;
        for (int j = 0; j <= lcpk::kMaxHLev; ++j) {
            x->hoff[j] = g->hoff[j];
            x->hlen[j] = g->hlen[j];
        }
        return launch_build_graph(g, x, d_tokens, f, N, s, huge);
    }
    g->sig_ok = false;
    const lcp_index_s saved = *x;
    (void)side_stream();  // created outside the capture
    LCP_CUDA_TRY(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
    int rc = build_sorted_ids(d_tokens, f, N, x->buf[0].ids, x->status, g->cap, huge, g->scratch);
    if (rc == LCP_OK && cudaEventRecordWithFlags(g->chk, g->cap, cudaEventRecordExternal) != cudaSuccess)
        rc = LCP_ERR_CUDA;
    if (rc == LCP_OK) rc = gather_rows_and_lcp(d_tokens, f, N, x->buf[0].ids, x->buf[0], x->W, g->cap);
    if (rc == LCP_OK) rc = build_aux(x, g->cap, false);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(g->cap, &graph);
    if (rc != LCP_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        *x = saved;
        cudaGetLastError();
        return LCP_PENDING;  // fall back to the direct path
    }
    if (g->exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(g->exec, graph, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(g->exec);
            g->exec = nullptr;
        }
    }
    if (!g->exec && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) {
        cudaGetLastError();
        g->exec = nullptr;
        cudaGraphDestroy(graph);
        *x = saved;
        return LCP_PENDING;
    }
    cudaGraphDestroy(graph);
    g->sig = sig;
    g->sig_ok = true;
    g->hlev = x->hlev;
    for (int j = 0; j <= lcpk::kMaxHLev; ++j) {
        g->hoff[j] = x->hoff[j];
        g->hlen[j] = x->hlen[j];
    }
    return launch_build_graph(g, x, d_tokens, f, N, s, huge);
}

static int alloc_index(lcp_index_s* x, int64_t N, int64_t cap, cudaStream_t s) {
    const int W = x->W;
    Carver c;  // every index array in one allocation
    int nsets = cap > N ? 2 : 1;
    for (int b = 0; b < nsets; ++b) {
        c.add(&x->buf[b].rows, (size_t)cap * W);
        c.add(&x->buf[b].head, (size_t)cap);
        c.add(&x->buf[b].ids, (size_t)cap);
        c.add(&x->buf[b].H, (size_t)cap);
    }
    c.add(&x->pos, (size_t)cap);
    c.add(&x->hmin, (size_t)(cap / 31 + 64));
    x->nblk_cap = (cap + lcpk::kBlk - 1) / lcpk::kBlk;
    if (x->nblk_cap < 1) x->nblk_cap = 1;
    c.add(&x->sblk, (size_t)x->nblk_cap * lcpk::kBlk);
    c.add(&x->soff, (size_t)x->nblk_cap * lcpk::kBlk);
    int lev = 0;
    while ((1ll << (lev + 1)) <= x->nblk_cap) ++lev;
    x->st_levels_cap = lev;
    c.add(&x->st, (size_t)(lev > 0 ? lev : 1) * x->nblk_cap * x->K);
    c.add(&x->bkt, ((size_t)1 << x->bits) + 1);
    c.add(&x->top, (size_t)lcpk::kTopLevels);
    if (cap == N && N >= lcpk::kSub2Min) {  // depth-2 tables: rebuilt by builds only
        c.add(&x->sub_idx, (size_t)1 << x->bits);
        c.add(&x->sub, (size_t)lcpk::kSub2Max << x->bits);
        c.add(&x->sub_count, 1);
    }
    // heavy-node tie lists: one table row per 128-row sample, one list per
    // node.  For max_k below kTieListMinK a tie fill from the sparse table
    // costs about as many loads as one from a list, so the lists (and their
    // rebuild on every insert) are left out and the search falls back to the
    // sparse table.
    c.add(&x->bkt_list, (size_t)1 << x->bits);
    if (x->max_k >= kTieListMinK) {
        x->nsamp_cap = (cap + lcpk::kBlk - 1) / lcpk::kBlk;
        if (x->nsamp_cap < 1) x->nsamp_cap = 1;
        const size_t nslots = (size_t)x->nsamp_cap * (size_t)(x->L + 1);
        x->nlists_cap = 4 * x->nsamp_cap + 64;
        c.add(&x->tbl, nslots);
        c.add(&x->slot_flag, nslots);
        c.add(&x->slot_lo, nslots);
        c.add(&x->slot_hi, nslots);
        c.add(&x->slot_list, nslots);
        c.add(&x->tl_sums, (nslots + 2047) / 2048);
        c.add(&x->tl_total, 4);
        c.add(&x->tlists, (size_t)x->nlists_cap * x->K);
        c.add(&x->tlpos, (size_t)x->nlists_cap * x->K);
        c.add(&x->tl_lo, (size_t)x->nlists_cap);
        c.add(&x->tl_hi, (size_t)x->nlists_cap);
    }
    c.add(&x->status, 1);
    if (cap > N) {
        c.add(&x->ins_rows, (size_t)2 * LCP_INSERT_SMALL_BATCH * W);
        c.add(&x->ins_ids, (size_t)LCP_INSERT_SMALL_BATCH);
        c.add(&x->ins_rank, (size_t)2 * LCP_INSERT_SMALL_BATCH);
    }
    LCP_CUDA_TRY(c.alloc(&x->arena, s));
    x->bytes = (int64_t)c.total;
    LCP_CUDA_TRY(cudaMemsetAsync(x->bkt_list, 0xFF, sizeof(int32_t) << x->bits, s));
    LCP_CUDA_TRY(cudaMemsetAsync(x->status, 0, sizeof(int), s));
    return LCP_OK;
}

// Reads and clears a device status word (s == nullptr: blocking copies).
static int read_status(int* d_status, cudaStream_t s) {
    if (!d_status) return LCP_OK;
    int h = 0;
    if (s) {
        LCP_CUDA_TRY(cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
        LCP_CUDA_TRY(cudaStreamSynchronize(s));
    } else {
        LCP_CUDA_TRY(cudaMemcpy(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost));
    }
    if (h) {
        LCP_CUDA_TRY(cudaMemset(d_status, 0, sizeof(int)));
        return h == lcpk::DEV_TIMEOUT ? LCP_ERR_TIMEOUT : LCP_ERR_CUDA;
    }
    return LCP_OK;
}

}  // namespace lcph

using namespace lcph;

namespace lcpk {
// Waits on a flag that nothing sets, at most `limit` spins, then reports.
__global__ void k_debug_wait(const volatile int* flag, long long limit, int* status) {
    long long spins = 0;
    while (*flag == 0) {
        if (++spins > limit) {
            flag_status(status, DEV_TIMEOUT);
            return;
        }
    }
}
}  // namespace lcpk

extern "C" {

const char* lcp_status_string(int s) {
    switch (s) {
        case LCP_OK: return "ok";
        case LCP_PENDING: return "pending";
        case LCP_ERR_INVALID: return "invalid argument";
        case LCP_ERR_OOM: return "device out of memory";
        case LCP_ERR_CAPACITY: return "index capacity exceeded";
        case LCP_ERR_BUDGET: return "request exceeds the session memory budget";
        case LCP_ERR_TIMEOUT: return "bounded wait timed out";
        case LCP_ERR_CUDA: return "CUDA error";
        case LCP_ERR_STATE: return "object in wrong state";
        default: return "unknown status";
    }
}

int lcp_index_build(const void* d_tokens, int64_t N, lcp_format_t fmt, int64_t capacity,
                    int32_t max_k, lcp_stream_t stream, lcp_index_t* out) {
    if (!out) return LCP_ERR_INVALID;
    *out = nullptr;
    if (!valid_build_fmt(fmt, max_k) || N < 0 || N >= (1ll << 30) || (N > 0 && !d_tokens)) return LCP_ERR_INVALID;
    if (max_k < 1 || max_k > LCP_INDEX_MAX_K) return LCP_ERR_INVALID;
    if (capacity == 0) capacity = N;
    if (capacity < N || capacity >= (1ll << 30)) return LCP_ERR_INVALID;
    if (fmt.L > LCP_MAX_L && capacity != N) return LCP_ERR_INVALID;  // wide rows: no inserts
    cudaStream_t s = (cudaStream_t)stream;
    lcp_index_s* x = new (std::nothrow) lcp_index_s();
    if (!x) return LCP_ERR_OOM;
    cudaGetDevice(&x->device);
    x->tb = fmt.token_bytes;
    x->L = fmt.L;
    x->vocab = fmt.vocab;
    x->tpw = 8 / x->tb;
    x->bits = 8 * x->tb;
    x->W = (x->L + x->tpw - 1) / x->tpw;
    x->max_k = max_k;
    x->K = ((max_k + 31) / 32) * 32;
    x->cap = capacity;
    x->N = N;
    retain_pool_memory();
    int rc = alloc_index(x, N, capacity, s);
    if (rc == LCP_OK && N > 1 && g_build_graph.load(std::memory_order_relaxed)) {
        // the usual path: the whole build replayed as one CUDA graph
        const int g = graph_build(x, d_tokens, N, s);
        if (g == LCP_OK) {
            note_use(x, s);
            *out = x;
            return LCP_OK;
        }
        if (g != LCP_PENDING) rc = g;  // LCP_PENDING: not graph-capturable here, build below
    }
    if (rc == LCP_OK && N > 0) {
        // Issued without waiting for the device.  Rows the on-device group
        // sort does not take (more than 2,048 rows sharing word 0, or a group
        // of 33-2,048 in which a row shares word 1 with more than 64 others)
        // need the exact (host-driven) refinement; their count lands in
        // pinned memory behind an event recorded mid-build, checked once
        // everything is queued -- by then
        // the device is usually past it, so the host returns while the
        // device still runs the tail of the build.  A nonzero count (rare:
        // heavy duplication) redoes the order exactly.
        lcpk::RowFmt f = lcpk::make_fmt(x->tb, x->L, d_tokens);
        uint32_t* huge = pinned_words() + 12;
        cudaEvent_t chk = nullptr;
        const bool fast = huge && cudaEventCreateWithFlags(&chk, cudaEventDisableTiming) == cudaSuccess;
        if (fast) {
            *huge = 0;
            rc = build_sorted_ids(d_tokens, f, N, x->buf[0].ids, x->status, s, huge);
            if (rc == LCP_OK) LCP_CUDA_TRY(cudaEventRecord(chk, s));
        } else {
            rc = build_sorted_ids(d_tokens, f, N, x->buf[0].ids, x->status, s);
        }
        if (rc == LCP_OK) rc = gather_rows_and_lcp(d_tokens, f, N, x->buf[0].ids, x->buf[0], x->W, s);
        if (rc == LCP_OK) rc = build_aux(x, s, false);
        if (fast) {
            if (rc == LCP_OK && cudaEventSynchronize(chk) == cudaSuccess && *huge != 0) {
                rc = build_sorted_ids(d_tokens, f, N, x->buf[0].ids, x->status, s);
                if (rc == LCP_OK) rc = gather_rows_and_lcp(d_tokens, f, N, x->buf[0].ids, x->buf[0], x->W, s);
                if (rc == LCP_OK) rc = build_aux(x, s, false);
            }
            cudaEventDestroy(chk);
        }
    }
    if (rc == LCP_OK) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_status(e);
    }
    if (rc != LCP_OK) {
        cudaStreamSynchronize(s);
        free_index_memory(x, s);
        cudaStreamSynchronize(s);
        delete x;
        return rc;
    }
    note_use(x, s);
    *out = x;
    return LCP_OK;
}

// The host-buffer entry points of this thread on the current device: device
// staging for queries and results (grown on demand, kept for the thread's
// later calls -- each call synchronises before it returns, so the next one
// finds them idle) and the event after this thread's latest host-to-device
// input copy.  A call's input copies wait for that event: the copies cross
// the link in call order, so a search's queries follow -- rather than share
// the link with -- the tokens of the build before it, yet overlap that build.
// The pipelined search also keeps its two copy streams and per-chunk events
// here.
constexpr int kHostChunks = 8;
struct HostStage {
    void* in = nullptr;
    size_t in_bytes = 0;
    void* out = nullptr;
    size_t out_bytes = 0;
    cudaEvent_t in_tail = nullptr;
    bool tail_set = false;
    cudaStream_t cin = nullptr, cout = nullptr;
    cudaEvent_t ev[2 * kHostChunks] = {nullptr};
};

static HostStage* host_stage() {
    static thread_local HostStage hs[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    HostStage& h = hs[dev];
    if (!h.in_tail) {
        bool ok = cudaEventCreateWithFlags(&h.in_tail, cudaEventDisableTiming) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&h.cin, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&h.cout, cudaStreamNonBlocking) == cudaSuccess;
        for (int i = 0; ok && i < 2 * kHostChunks; ++i)
            ok = cudaEventCreateWithFlags(&h.ev[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            h = HostStage();  // (a partial set is leaked, not reused)
            return nullptr;
        }
    }
    return &h;
}

// Device buffer of at least `need` bytes (synchronous allocation, usable from
// any stream at once; the old buffer is idle when this is called).
static int grow(void** p, size_t* have, size_t need) {
    if (*have >= need) return LCP_OK;
    if (*p) {
        cudaFree(*p);
        *p = nullptr;
        *have = 0;
    }
    LCP_CUDA_TRY(cudaMalloc(p, need));
    *have = need;
    return LCP_OK;
}

int lcp_index_build_host(const void* h_tokens, int64_t N, lcp_format_t fmt, int64_t capacity,
                         int32_t max_k, lcp_stream_t stream, lcp_index_t* out) {
    if (!out) return LCP_ERR_INVALID;
    *out = nullptr;
    if (!valid_build_fmt(fmt, max_k) || N < 0 || N >= (1ll << 30) || (N > 0 && !h_tokens)) return LCP_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = (size_t)N * fmt.L * fmt.token_bytes;
    void* d = nullptr;
    if (bytes) {
        HostStage* hs = host_stage();
        LCP_CUDA_TRY(cudaMallocAsync(&d, bytes, s));
        if (hs && hs->tail_set) LCP_CUDA_TRY(cudaStreamWaitEvent(s, hs->in_tail, 0));
        LCP_CUDA_TRY(cudaMemcpyAsync(d, h_tokens, bytes, cudaMemcpyHostToDevice, s));
        if (hs && cudaEventRecord(hs->in_tail, s) == cudaSuccess) hs->tail_set = true;
    }
    int rc = lcp_index_build(d, N, fmt, capacity, max_k, stream, out);
    if (d) cudaFreeAsync(d, s);
    return rc;
}

int lcp_index_insert(lcp_index_t x, const void* d_tokens, int64_t n, lcp_stream_t stream) {
    if (!x || n < 0 || (n > 0 && !d_tokens) || index_is_wide(x)) return LCP_ERR_INVALID;
    if (n == 0) return LCP_OK;
    if (x->N + n > x->cap) return LCP_ERR_CAPACITY;
    if (!x->buf[1].rows) return LCP_ERR_CAPACITY;
    int rc = insert_device(x, d_tokens, n, (cudaStream_t)stream);
    if (rc == LCP_OK) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_status(e);
    }
    note_use(x, (cudaStream_t)stream);
    return rc;
}

int lcp_topk_batch(lcp_index_t x, const void* d_queries, int64_t Q, int32_t k, int32_t* d_out_ids,
                   uint8_t* d_out_lcp, lcp_stream_t stream) {
    if (!x || Q < 0 || k < 1 || k > x->max_k || index_is_wide(x)) return LCP_ERR_INVALID;
    if (Q > 0 && (!d_queries || !d_out_ids || !d_out_lcp)) return LCP_ERR_INVALID;
    int rc = topk_batch_device(x, d_queries, Q, k, d_out_ids, d_out_lcp, (cudaStream_t)stream);
    if (rc == LCP_OK) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_status(e);
    }
    note_use(x, (cudaStream_t)stream);
    return rc;
}

int lcp_topk_batch_host(lcp_index_t x, const void* h_queries, int64_t Q, int32_t k, int32_t* h_out_ids,
                        uint8_t* h_out_lcp, lcp_stream_t stream) {
    if (!x || Q < 0 || k < 1 || k > x->max_k || index_is_wide(x)) return LCP_ERR_INVALID;
    if (Q == 0) return LCP_OK;
    if (!h_queries || !h_out_ids || !h_out_lcp) return LCP_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t row = (size_t)x->L * x->tb;
    size_t qb = (size_t)Q * row;
    size_t ob = (size_t)Q * k * (sizeof(int32_t) + 1);
    int rc;
    HostStage* hs = host_stage();
    if (!hs) return LCP_ERR_CUDA;
    if ((rc = grow(&hs->in, &hs->in_bytes, qb))) return rc;
    if ((rc = grow(&hs->out, &hs->out_bytes, ob))) return rc;
    int32_t* d_ids = (int32_t*)hs->out;
    uint8_t* d_lcp = (uint8_t*)hs->out + (size_t)Q * k * sizeof(int32_t);
    const uint8_t* hq = static_cast<const uint8_t*>(h_queries);
    uint8_t* dq = static_cast<uint8_t*>(hs->in);
    // Pipelined in chunks: chunk i's queries cross the bus on one copy
    // stream while chunk i-1 is searched on `stream` and chunk i-2's results
    // cross back on another, so the two directions and the search overlap.
    const int64_t chunk = Q >= kHostChunks * 65536 ? (Q + kHostChunks - 1) / kHostChunks : Q;
    const int nch = (int)((Q + chunk - 1) / chunk);
    cudaStream_t cin = hs->cin, cout = hs->cout;
    cudaEvent_t* ev = hs->ev;
    cudaError_t e = cudaSuccess;
    // the input copies follow this thread's earlier ones (not the whole stream)
    if (nch > 1 && hs->tail_set) e = cudaStreamWaitEvent(cin, hs->in_tail, 0);
    if (e != cudaSuccess) return cuda_status(e);
    for (int i = 0; i < nch && rc == LCP_OK; ++i) {
        const int64_t q0 = i * chunk, qc = q0 + chunk < Q ? chunk : Q - q0;
        cudaStream_t in = nch > 1 ? cin : s, out = nch > 1 ? cout : s;
        if (nch == 1 && hs->tail_set) e = cudaStreamWaitEvent(in, hs->in_tail, 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dq + q0 * row, hq + q0 * row, qc * row, cudaMemcpyHostToDevice, in);
        if (e == cudaSuccess && i == nch - 1 && cudaEventRecord(hs->in_tail, in) == cudaSuccess) hs->tail_set = true;
        if (e == cudaSuccess && nch > 1) {
            e = cudaEventRecord(ev[2 * i], in);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[2 * i], 0);
        }
        if (e != cudaSuccess) {
            rc = cuda_status(e);
            break;
        }
        rc = lcp_topk_batch(x, dq + q0 * row, qc, k, d_ids + q0 * k, d_lcp + q0 * k, stream);
        if (rc != LCP_OK) break;
        if (nch > 1) {
            e = cudaEventRecord(ev[2 * i + 1], s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(out, ev[2 * i + 1], 0);
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_out_ids + q0 * k, d_ids + q0 * k, (size_t)qc * k * sizeof(int32_t),
                                cudaMemcpyDeviceToHost, out);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_out_lcp + q0 * k, d_lcp + q0 * k, (size_t)qc * k, cudaMemcpyDeviceToHost, out);
        if (e != cudaSuccess) rc = cuda_status(e);
    }
    if (nch > 1) {
        cudaStreamSynchronize(cin);
        cudaStreamSynchronize(cout);
    }
    cudaStreamSynchronize(s);
    return rc;
}

int lcp_scan_topk(const void* d_tokens, int64_t N, lcp_format_t fmt, const void* d_queries, int64_t Q,
                  int32_t k, int32_t* d_out_ids, uint8_t* d_out_lcp, lcp_stream_t stream) {
    if (!valid_fmt(fmt) || N < 0 || N >= (1ll << 30) || Q < 0 || k < 1 || k > LCP_SCAN_MAX_K)
        return LCP_ERR_INVALID;
    if (Q > 0 && (!d_queries || !d_out_ids || !d_out_lcp)) return LCP_ERR_INVALID;
    if (N > 0 && Q > 0 && !d_tokens) return LCP_ERR_INVALID;
    retain_pool_memory();  // per-call scratch comes from the pool: keep it mapped between calls
    int rc = scan_topk_device(d_tokens, N, fmt.token_bytes, fmt.L, d_queries, Q, k, d_out_ids,
                              d_out_lcp, (cudaStream_t)stream);
    if (rc == LCP_OK) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_status(e);
    }
    return rc;
}

int lcp_index_size(lcp_index_t x, int64_t* N, int64_t* bytes) {
    if (!x) return LCP_ERR_INVALID;
    if (N) *N = x->N;
    if (bytes) *bytes = x->bytes;
    return LCP_OK;
}

int lcp_index_export(lcp_index_t x, int32_t* d_ids, uint8_t* d_H, lcp_stream_t stream) {
    if (!x || (d_H && index_is_wide(x))) return LCP_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    if (x->N == 0) return LCP_OK;
    if (d_ids)
        LCP_CUDA_TRY(cudaMemcpyAsync(d_ids, x->buf[x->cur].ids, sizeof(int32_t) * x->N,
                                     cudaMemcpyDeviceToDevice, s));
    if (d_H)
        LCP_CUDA_TRY(cudaMemcpyAsync(d_H, x->buf[x->cur].H, (size_t)x->N, cudaMemcpyDeviceToDevice, s));
    note_use(x, s);
    return LCP_OK;
}

int lcp_index_sync(lcp_index_t x) {
    if (!x) return LCP_ERR_INVALID;
    if (x->shared) LCP_CUDA_TRY(cudaDeviceSynchronize());
    for (int i = 0; i < x->nuses; ++i) LCP_CUDA_TRY(cudaEventSynchronize(x->uses[i].e));
    return read_status(x->status, nullptr);
}

int lcp_index_destroy(lcp_index_t x) {
    if (!x) return LCP_OK;
    if (x->shared) {
        // held by a session or work queue, or used on many streams: wait
        // for the whole device, then free
        cudaDeviceSynchronize();
        free_index_memory(x, nullptr);
    } else {
        // stream-ordered: the frees wait (on the library's free stream) for
        // the last operation on every stream the index was used on; the
        // host does not wait.  Events, not streams, are waited on, so a
        // stream destroyed by its owner meanwhile does not matter.
        cudaStream_t fs = free_stream();
        for (int i = 0; i < x->nuses; ++i) cudaStreamWaitEvent(fs, x->uses[i].e, 0);
        free_index_memory(x, fs);
    }
    for (int i = 0; i < x->nuses; ++i) cudaEventDestroy(x->uses[i].e);
    delete x;
    return LCP_OK;
}

int lcp_device_status(void) {
    LCP_CUDA_TRY(cudaDeviceSynchronize());
    return read_status(lib_status_word(), 0);
}

int64_t lcp_launch_count(void) { return g_launches.load(); }

int lcp_kernel_timing(int enable) {
    std::lock_guard<std::mutex> lk(g_kt_mu);
    if (enable) {
        for (auto& r : g_kt_pending) {
            cudaEventSynchronize(r.b);
            g_kt_pool.push_back(r.a);
            g_kt_pool.push_back(r.b);
        }
        g_kt_pending.clear();
        g_kt_total.clear();
    }
    g_kt_on.store(enable != 0);
    return LCP_OK;
}

int lcp_build_graph(int enable) {
    g_build_graph.store(enable != 0);
    return LCP_OK;
}

int lcp_kernel_timing_filter(const char* prefix) {
    std::lock_guard<std::mutex> lk(g_kt_mu);
    g_kt_filter = prefix ? prefix : "";
    return LCP_OK;
}

int lcp_kernel_time(const char* prefix, double* total_ms, int64_t* launches) {
    if (!prefix) return LCP_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_kt_mu);
    for (auto& r : g_kt_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            auto& t = g_kt_total[r.name];
            t.first += ms;
            t.second += 1;
        }
        g_kt_pool.push_back(r.a);
        g_kt_pool.push_back(r.b);
    }
    g_kt_pending.clear();
    double ms = 0;
    int64_t n = 0;
    const size_t len = strlen(prefix);
    for (auto& kv : g_kt_total)
        if (kv.first.compare(0, len, prefix) == 0) {
            ms += kv.second.first;
            n += kv.second.second;
        }
    if (total_ms) *total_ms = ms;
    if (launches) *launches = n;
    return LCP_OK;
}

int lcp_debug_bounded_wait(int64_t spin_limit, lcp_stream_t stream) {
    if (spin_limit < 1) return LCP_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    int* flag = nullptr;
    int* st = nullptr;
    LCP_CUDA_TRY(cudaMallocAsync((void**)&flag, sizeof(int), s));
    LCP_CUDA_TRY(cudaMallocAsync((void**)&st, sizeof(int), s));
    LCP_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), s));
    LCP_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(int), s));
    LCP_LAUNCH(lcpk::k_debug_wait, 1, 1, 0, s, flag, (long long)spin_limit, st);
    int rc = read_status(st, s);
    cudaFreeAsync(flag, s);
    cudaFreeAsync(st, s);
    cudaStreamSynchronize(s);
    return rc;
}

}  // extern "C"
