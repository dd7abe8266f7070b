// Streaming insert-then-query step replayed as a CUDA graph (see lcp.h).
//
// The step's host code is the same as lcp_index_insert + lcp_topk_batch; run
// under stream capture it records the kernels instead of launching them.  The
// index's host-side fields (N, buffer parity, tree levels) advance during the
// capture exactly as they would for a direct call, and are restored if the
// capture fails.  Successive steps differ only in kernel arguments and grid
// sizes (N grows), which cudaGraphExecUpdate applies to the instantiated
// graph; a change in the number of kernels forces a new instantiation.
#include <new>

#include "index.cuh"

struct lcp_step_s {
    lcp_index_s* x = nullptr;
    int64_t n = 0, Q = 0;
    int k = 0;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    void* loc = nullptr;  // search scratch (a captured graph must not allocate)
    int64_t runs = 0, inst = 0;
};

extern "C" {

int lcp_step_create(lcp_index_t x, int64_t n, int64_t Q, int32_t k, lcp_step_t* out) {
    if (!x || !out || n < 0 || n > LCP_INSERT_SMALL_BATCH || Q < 0 || k < 1 || k > x->max_k ||
        lcph::index_is_wide(x))
        return LCP_ERR_INVALID;
    *out = nullptr;
    lcp_step_s* st = new (std::nothrow) lcp_step_s();
    if (!st) return LCP_ERR_OOM;
    st->x = x;
    st->n = n;
    st->Q = Q;
    st->k = k;
    lcph::sm_count();  // cache the device attribute outside any capture
    cudaError_t e = cudaStreamCreateWithFlags(&st->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&st->loc, lcph::search_scratch_bytes(Q));
    if (e != cudaSuccess) {
        if (st->cap) cudaStreamDestroy(st->cap);
        delete st;
        return lcph::cuda_status(e);
    }
    *out = st;
    return LCP_OK;
}

int lcp_step_run(lcp_step_t st, const void* d_insert, const void* d_queries, int32_t* d_out_ids,
                 uint8_t* d_out_lcp, lcp_stream_t stream) {
    if (!st) return LCP_ERR_INVALID;
    lcp_index_s* x = st->x;
    if ((st->n > 0 && !d_insert) || (st->Q > 0 && (!d_queries || !d_out_ids || !d_out_lcp)))
        return LCP_ERR_INVALID;
    if (st->n > 0 && (x->N + st->n > x->cap || !x->buf[1].rows)) return LCP_ERR_CAPACITY;
    const lcp_index_s saved = *x;  // host-side state, restored if capture fails
    const int64_t before = lcp_launch_count();
    (void)lcph::side_stream();  // created outside the capture
    LCP_CUDA_TRY(cudaStreamBeginCapture(st->cap, cudaStreamCaptureModeThreadLocal));
    int rc = st->n > 0 ? lcph::insert_device(x, d_insert, st->n, st->cap) : LCP_OK;
    if (rc == LCP_OK && st->Q > 0)
        rc = lcph::topk_batch_device(x, d_queries, st->Q, st->k, d_out_ids, d_out_lcp, st->cap, st->loc);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st->cap, &g);
    // kernels recorded, not launched: counted when the graph runs (the
    // count is process-wide, so launches by other threads meanwhile blur it)
    const int64_t nodes = lcp_launch_count() - before;
    lcph::count_launch(-(int)nodes);
    if (rc == LCP_OK && e != cudaSuccess) rc = lcph::cuda_status(e);
    if (rc != LCP_OK) {
        if (g) cudaGraphDestroy(g);
        *x = saved;
        cudaGetLastError();
        return rc;
    }
    if (st->exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(st->exec, g, &info) != cudaSuccess) {
            cudaGetLastError();  // refused: instantiate anew below
            cudaGraphExecDestroy(st->exec);
            st->exec = nullptr;
        }
    }
    if (!st->exec) {
        e = cudaGraphInstantiate(&st->exec, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            *x = saved;
            return lcph::cuda_status(e);
        }
        st->inst++;
    }
    cudaGraphDestroy(g);
    LCP_CUDA_TRY(cudaGraphLaunch(st->exec, (cudaStream_t)stream));
    lcph::count_launch((int)nodes);
    lcph::note_use(x, (cudaStream_t)stream);
    st->runs++;
    return LCP_OK;
}

int lcp_step_stats(lcp_step_t st, int64_t* runs, int64_t* instantiations) {
    if (!st) return LCP_ERR_INVALID;
    if (runs) *runs = st->runs;
    if (instantiations) *instantiations = st->inst;
    return LCP_OK;
}

int lcp_step_destroy(lcp_step_t st) {
    if (!st) return LCP_OK;
    cudaDeviceSynchronize();
    if (st->exec) cudaGraphExecDestroy(st->exec);
    cudaFree(st->loc);
    cudaStreamDestroy(st->cap);
    delete st;
    return LCP_OK;
}

}  // extern "C"
