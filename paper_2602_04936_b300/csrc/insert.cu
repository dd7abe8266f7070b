// Insertion of a batch of rows into a built index.  The paper's analysis is
// static (Sec. 10.1, App. G); this extends Algorithm 1 so that the result is
// exactly BuildLCPIndex of the concatenated dataset.
//
//   1. the batch is packed and sorted: rank sort for small batches (no host
//      round trip, so a streaming step can be captured in a CUDA graph),
//      the build's radix sort otherwise;
//   2. every sorted new row finds its merge-path position: the number of old
//      rows <= it (equal old rows have smaller ids and come first) plus its
//      rank in the batch;
//   3. one pass writes the merged rows / head / ids into the spare buffer
//      set: an output slot is new iff it is one of those positions, else it
//      takes the next old row;
//   4. H is recomputed over the merged rows and the tie tables rebuilt.
#include "index.cuh"

namespace lcpk {

__global__ void k_ins_pack(const uint8_t* __restrict__ tokens, RowFmt f, int64_t n, int W,
                           uint64_t* __restrict__ out) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * W) return;
    int64_t r = e / W;
    int w = (int)(e - r * W);
    out[e] = pack_word(row_of(tokens, r, f), w, f);
}

__device__ __forceinline__ int cmp_rows(const uint64_t* a, const uint64_t* b, int W) {
    for (int w = 0; w < W; ++w) {
        if (a[w] != b[w]) return a[w] < b[w] ? -1 : 1;
    }
    return 0;
}

// rank[i] = number of batch rows ordered before row i (row, then batch index).
__global__ void k_ins_rank(const uint64_t* __restrict__ rows, int n, int W,
                           int32_t* __restrict__ order) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t* me = rows + (int64_t)i * W;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
        int c = cmp_rows(rows + (int64_t)j * W, me, W);
        rank += (c < 0) || (c == 0 && j < i);
    }
    order[rank] = i;
}

// Sorted new rows and ids (id = N + batch index).
__global__ void k_ins_sorted(const uint64_t* __restrict__ rows, const int32_t* __restrict__ order,
                             int64_t n, int W, int64_t N, uint64_t* __restrict__ srows,
                             int32_t* __restrict__ sids) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * W) return;
    int64_t j = e / W;
    int w = (int)(e - j * W);
    int32_t src = order[j];
    srows[e] = rows[(int64_t)src * W + w];
    if (w == 0) sids[j] = (int32_t)(N + src);
}

// np[j] = j + #{old rows <= new row j}.
__global__ void k_ins_locate(const uint64_t* __restrict__ old_rows, const uint64_t* __restrict__ old_head,
                             int64_t N, const uint64_t* __restrict__ srows, int64_t n, int W,
                             int64_t* __restrict__ np) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint64_t* me = srows + j * W;
    int64_t lo = 0, hi = N;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        int c;
        if (old_head[mid] != me[0]) c = old_head[mid] < me[0] ? -1 : 1;
        else c = cmp_rows(old_rows + mid * W, me, W);
        if (c <= 0) lo = mid + 1;
        else hi = mid;
    }
    np[j] = j + lo;
}

// One thread per output word: slot o is new row j if np[j] == o, else old row
// o - #{np < o}.
__global__ void k_ins_merge(const uint64_t* __restrict__ old_rows, const int32_t* __restrict__ old_ids,
                            const uint64_t* __restrict__ srows, const int32_t* __restrict__ sids,
                            const int64_t* __restrict__ np, int64_t n, int64_t total, int W,
                            uint64_t* __restrict__ rows, uint64_t* __restrict__ head,
                            int32_t* __restrict__ ids) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total * W) return;
    int64_t o = e / W;
    int w = (int)(e - o * W);
    int64_t lo = 0, hi = n;  // #{np < o}
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (np[mid] < o) lo = mid + 1;
        else hi = mid;
    }
    uint64_t x;
    int32_t id;
    if (lo < n && np[lo] == o) {
        x = srows[lo * W + w];
        id = sids[lo];
    } else {
        int64_t i = o - lo;
        x = old_rows[i * W + w];
        id = old_ids[i];
    }
    rows[e] = x;
    if (w == 0) {
        head[o] = x;
        ids[o] = id;
    }
}

}  // namespace lcpk

namespace lcph {
using namespace lcpk;

static inline unsigned nblocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

int insert_device(lcp_index_s* x, const void* d_tokens, int64_t n, cudaStream_t s) {
    if (n <= 0) return LCP_OK;
    const int W = x->W;
    RowFmt f = make_fmt(x->tb, x->L, d_tokens);
    const bool small = n <= LCP_INSERT_SMALL_BATCH;
    uint64_t* packed = nullptr;
    uint64_t* srows = x->ins_rows;
    int32_t* sids = x->ins_ids;
    int32_t* order = nullptr;
    int64_t* np = x->ins_rank;
    bool own = !small;
    if (own) {
        LCP_CUDA_TRY(cudaMallocAsync((void**)&srows, sizeof(uint64_t) * n * W, s));
        LCP_CUDA_TRY(cudaMallocAsync((void**)&sids, sizeof(int32_t) * n, s));
        LCP_CUDA_TRY(cudaMallocAsync((void**)&np, sizeof(int64_t) * n, s));
        LCP_CUDA_TRY(cudaMallocAsync((void**)&order, sizeof(int32_t) * n, s));
        LCP_CUDA_TRY(cudaMallocAsync((void**)&packed, sizeof(uint64_t) * n * W, s));
    } else {
        order = reinterpret_cast<int32_t*>(x->ins_rank + LCP_INSERT_SMALL_BATCH);
        packed = x->ins_rows + (int64_t)LCP_INSERT_SMALL_BATCH * W;
    }
    int rc = LCP_OK;
    LCP_LAUNCH(k_ins_pack, nblocks(n * W, 256), 256, 0, s, reinterpret_cast<const uint8_t*>(d_tokens),
               f, n, W, packed);
    if (small) {
        LCP_LAUNCH(k_ins_rank, nblocks(n, 128), 128, 0, s, packed, (int)n, W, order);
    } else {
        rc = build_sorted_ids(d_tokens, f, n, order, x->status, s);
    }
    if (rc == LCP_OK) {
        LCP_LAUNCH(k_ins_sorted, nblocks(n * W, 256), 256, 0, s, packed, order, n, W, x->N, srows,
                   sids);
        lcp_buffers& ob = x->buf[x->cur];
        lcp_buffers& nb = x->buf[1 - x->cur];
        LCP_LAUNCH(k_ins_locate, nblocks(n, 128), 128, 0, s, ob.rows, ob.head, x->N, srows, n, W, np);
        const int64_t total = x->N + n;
        LCP_LAUNCH(k_ins_merge, nblocks(total * W, 256), 256, 0, s, ob.rows, ob.ids, srows, sids, np,
                   n, total, W, nb.rows, nb.head, nb.ids);
        rc = adjacent_lcp(nb.rows, total, W, x->L, x->tpw, x->bits, nb.H, s);
        if (rc == LCP_OK) {
            x->cur = 1 - x->cur;
            x->N = total;
            rc = build_aux(x, s);
        }
    }
    if (own) {
        cudaFreeAsync(srows, s);
        cudaFreeAsync(sids, s);
        cudaFreeAsync(np, s);
        cudaFreeAsync(order, s);
        cudaFreeAsync(packed, s);
    }
    return rc;
}

}  // namespace lcph
