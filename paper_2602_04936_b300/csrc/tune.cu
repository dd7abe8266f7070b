// Autotuner for the indexed search's launch shape.
//
// The shape -- one fused kernel (a warp per query), or locate + answer +
// fill with some queries per warp for the answer and queries located one per
// lane or one per warp -- changes only the schedule, never a result.  The tuner times every candidate on the caller's sample
// batch with CUDA events (one warm-up run, best of three) and records the
// fastest in a process-wide table keyed by the index's shape class
// (log2 N, L, token bytes) and the batch's (log2 Q, k class); later searches
// of that class use it.  Tuned entries can be read back and installed again
// (lcp_set_search_shape), so a tuning run can be cached across processes.
#include "search.cuh"

extern "C" {

int lcp_autotune(lcp_index_t x, const void* d_queries, int64_t Q, int32_t k, lcp_stream_t stream,
                 lcp_tune_result_t* best) {
    if (!x || !d_queries || Q < 1 || k < 1 || k > x->max_k || !best || lcph::index_is_wide(x))
        return LCP_ERR_INVALID;
    if (x->N == 0) return LCP_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t* ids = nullptr;
    uint8_t* lcp = nullptr;
    void* loc = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&ids, sizeof(int32_t) * (size_t)Q * k, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&lcp, (size_t)Q * k, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&loc, lcph::search_scratch_bytes(Q), s);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    int rc = e == cudaSuccess ? LCP_OK : lcph::cuda_status(e);
    auto time_shape = [&](const lcph::SearchShape& sh, float* ms) -> int {
        float bestms = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(a, s);
            int r = lcph::topk_batch_device(x, d_queries, Q, k, ids, lcp, s, loc, &sh);
            if (r != LCP_OK) return r;
            cudaEventRecord(b, s);
            cudaError_t ee = cudaEventSynchronize(b);
            if (ee != cudaSuccess) return lcph::cuda_status(ee);
            float t = 0.f;
            cudaEventElapsedTime(&t, a, b);
            if (rep > 0 && t < bestms) bestms = t;  // the first run warms up
        }
        *ms = bestms;
        return LCP_OK;
    };
    lcph::SearchShape chosen = lcph::default_shape(Q);
    float dflt = 0.f, top = 0.f;
    if (rc == LCP_OK) rc = time_shape(chosen, &dflt);
    top = dflt;
    for (int lw = 0; lw < 3 && rc == LCP_OK; ++lw) {  // lane, warp, lane over the staged top levels
        for (int qpw = 1; qpw <= 32 && rc == LCP_OK; qpw <<= 1) {
            lcph::SearchShape sh;
            sh.qpw = qpw;
            sh.locate_warp = lw;
            float t = 0.f;
            rc = time_shape(sh, &t);
            if (rc == LCP_OK && t < top) {
                top = t;
                chosen = sh;
            }
        }
    }
    if (rc == LCP_OK && !chosen.fused) {  // the fused kernel, for batches that use three by default
        lcph::SearchShape sh;
        sh.fused = 1;
        float t = 0.f;
        rc = time_shape(sh, &t);
        if (rc == LCP_OK && t < top) {
            top = t;
            chosen = sh;
        }
    }
    if (rc == LCP_OK) {
        lcph::set_search_shape(x, Q, k, chosen);
        best->qpw = chosen.fused ? 0 : chosen.qpw;
        best->locate_warp = chosen.locate_warp;
        best->best_ms = top;
        best->default_ms = dflt;
    }
    cudaFreeAsync(ids, s);
    cudaFreeAsync(lcp, s);
    cudaFreeAsync(loc, s);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    return rc;
}

int lcp_set_search_shape(lcp_index_t x, int64_t Q, int32_t k, int32_t qpw, int32_t locate_warp) {
    if (!x || Q < 1 || k < 1 || qpw < 0 || qpw > 32 || locate_warp < 0 || locate_warp > 2 ||
        lcph::index_is_wide(x))
        return LCP_ERR_INVALID;
    lcph::SearchShape sh;
    sh.fused = qpw == 0 ? 1 : 0;
    sh.qpw = qpw == 0 ? 1 : qpw;
    sh.locate_warp = locate_warp;
    lcph::set_search_shape(x, Q, k, sh);
    return LCP_OK;
}

}  // extern "C"
