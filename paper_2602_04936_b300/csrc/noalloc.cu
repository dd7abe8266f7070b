// Full scan top-k that allocates nothing.
//
// Some callers cannot allocate device memory when they call in: a real-time
// control loop (the paper's guidance/navigation example) must not block in
// the allocator, whose calls can synchronise the device and have no latency
// bound; code written to rules that allow allocation only at start-up; and
// host code issuing work inside a stream capture in global mode, where
// cudaMalloc is not permitted.  lcp_scan_topk takes its temporaries from the
// stream-ordered allocator; this entry point instead runs its per-thread-heap
// kernels (for every batch size, also where lcp_scan_topk would take the
// small-batch threshold selection) on a fixed scratch array that lives in the
// library's device image.  The results are the same bytes.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds it (LCP_SCAN_NOALLOC_SCRATCH_BYTES) until the process exits.
// Host code cannot use its name as a device address; the address is looked
// up once per device with cudaGetSymbolAddress on the first call made on
// that device.
#include <mutex>

#include "scan.cuh"

namespace {

static __device__ __align__(256) unsigned char g_scan_scratch[LCP_SCAN_NOALLOC_SCRATCH_BYTES];

struct ScratchSlot {
    std::mutex mu;
    void* ptr = nullptr;
};
ScratchSlot g_slots[64];

// Device address of g_scan_scratch on the current device.  Looked up on the
// first call per device; only a successful lookup is kept, so a call that
// failed (for example one made inside a global-mode stream capture) does not
// stop a later call from trying again.
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    ScratchSlot& s = g_slots[dev];
    std::lock_guard<std::mutex> lk(s.mu);
    if (!s.ptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scan_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
        s.ptr = p;
    }
    *out = s.ptr;
    return cudaSuccess;
}

}  // namespace

extern "C" int lcp_scan_topk_noalloc(const void* d_tokens, int64_t N, lcp_format_t fmt,
                                     const void* d_queries, int64_t Q, int32_t k, int32_t* d_out_ids,
                                     uint8_t* d_out_lcp, lcp_stream_t stream) {
    using namespace lcpk;
    if ((fmt.token_bytes != 1 && fmt.token_bytes != 2) || fmt.L < 1 || fmt.L > LCP_MAX_L || N < 0 ||
        N >= (1ll << 30) || Q < 0 || k < 1 || k > LCP_SCAN_MAX_K)
        return LCP_ERR_INVALID;
    if (Q > 0 && (!d_queries || !d_out_ids || !d_out_lcp)) return LCP_ERR_INVALID;
    if (N > 0 && Q > 0 && !d_tokens) return LCP_ERR_INVALID;
    if (Q == 0) return LCP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (N == 0) {
        LCP_CUDA_TRY(cudaMemsetAsync(d_out_ids, 0xFF, sizeof(int32_t) * (size_t)Q * k, s));
        LCP_CUDA_TRY(cudaMemsetAsync(d_out_lcp, 0, (size_t)Q * k, s));
        return LCP_OK;
    }
    // Scratch layout: [plane 0: N upper halves][N lower halves][counts: S x
    // Q][lists: S x Q x (k + kLogSlack) keys], each part starting on a
    // 256-byte boundary.  The batch
    // is scanned in its own order (no sort, no floor pass: those would need
    // more scratch); the results are the same bytes.
    const uint64_t cap = (uint64_t)LCP_SCAN_NOALLOC_SCRATCH_BYTES;
    const uint64_t half_bytes = ((uint64_t)N * 4 + 255) & ~255ull;  // each half of the plane
    const uint64_t plane_bytes = 2 * half_bytes;
    const int lcap = k + kLogSlack;  // log entries per (slice, query)
    auto need = [&](int64_t S) {
        return plane_bytes + (((uint64_t)S * Q * 4 + 255) & ~255ull) + (uint64_t)S * Q * lcap * 8;
    };
    if (need(1) > cap) return LCP_ERR_INVALID;  // too large even with one slice
    const int64_t qtiles = (Q + kScanPartialThreads - 1) / kScanPartialThreads;
    int64_t S = (148 * 4 + qtiles - 1) / qtiles;
    const int64_t maxS = (N + 1023) / 1024;
    if (S > maxS) S = maxS;
    if (S > kMergeMaxLists) S = kMergeMaxLists;
    while (S > 1 && need(S) > cap) --S;
    if (S < 1) S = 1;
    const int64_t slice = ((N + S - 1) / S + kScanSliceAlign - 1) / kScanSliceAlign * kScanSliceAlign;
    S = (N + slice - 1) / slice;

    void* base = nullptr;
    LCP_CUDA_TRY(scratch_address(&base));
    unsigned char* b = reinterpret_cast<unsigned char*>(base);
    uint32_t* plane_hi = reinterpret_cast<uint32_t*>(b);
    uint32_t* plane_lo = reinterpret_cast<uint32_t*>(b + half_bytes);
    int32_t* counts = reinterpret_cast<int32_t*>(b + plane_bytes);
    uint64_t* lists = reinterpret_cast<uint64_t*>(b + plane_bytes + (((uint64_t)S * Q * 4 + 255) & ~255ull));
    // Nothing in the scratch needs to start at zero: plane 0 is written in
    // full by the pack kernel, every count and every log slot the merge reads
    // by the scan kernel.  Calls that overlap on the GPU share the array and
    // race; callers must order them (one stream, or events).
    RowFmt f = make_fmt(fmt.token_bytes, fmt.L, d_tokens);
    RowFmt qf = make_fmt(fmt.token_bytes, fmt.L, d_queries);
    LCP_LAUNCH(k_pack_plane0, (unsigned)((N + 255) / 256), 256, 0, s,
               reinterpret_cast<const uint8_t*>(d_tokens), f, N, plane_hi, plane_lo);
    ScanArgs a;
    a.tokens = reinterpret_cast<const uint8_t*>(d_tokens);
    a.plane_hi = plane_hi;
    a.plane_lo = plane_lo;
    a.f = f;
    a.N = N;
    a.queries = reinterpret_cast<const uint8_t*>(d_queries);
    a.qf = qf;
    a.Q = Q;
    a.order = nullptr;
    a.floor = nullptr;
    a.k = k;
    a.cap = lcap;
    a.slice = slice;
    a.lists = lists;
    a.counts = counts;
    // the library's status word if some call made it already (this entry
    // point allocates nothing); a bounded wait that ran out is recorded there
    a.status = lcph::lib_status_word_if_any();
    LCP_LAUNCH(k_scan_partial, dim3((unsigned)qtiles, (unsigned)S), kScanPartialThreads, 0, s, a);
    LCP_CUDA_TRY(cudaFuncSetAttribute(k_scan_merge, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(sizeof(uint64_t) * kMergeCap)));
    LCP_LAUNCH(k_scan_merge, (unsigned)Q, 256, sizeof(uint64_t) * kMergeCap, s, lists, counts, lcap, Q, (int)S, k,
               (const int32_t*)nullptr, d_out_ids, d_out_lcp);
    LCP_CUDA_TRY(cudaGetLastError());
    return LCP_OK;
}
