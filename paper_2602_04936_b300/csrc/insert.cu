// Insertion of a batch of rows into a built index.  The paper's analysis is
// static (Sec. 10.1, App. G); this extends Algorithm 1 so that the result is
// exactly BuildLCPIndex of the concatenated dataset.
//
//   1. the batch is sorted and every new row finds its merge-path position:
//      the number of old rows <= it (equal old rows have smaller ids and
//      come first) plus its rank in the batch.  Small batches do both in one
//      warp-per-row kernel with no host round trip (so a streaming step can
//      be captured in a CUDA graph); large ones use the build's radix sort
//      and a binary search per row;
//   2. one pass writes the merged rows / head / ids / H / pos into the spare
//      buffer set (an output slot is new iff it is one of those positions,
//      else it takes the next old row; H is only recomputed next to new
//      rows) and shifts the depth-1 bucket table;
//   3. the min tree, sorted blocks, sparse table and tie lists are rebuilt.
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

// Compares raw batch row a with batch row b (whose word 0 is b0), packing
// words on the fly; words past 0 are only packed on a tie.
__device__ __forceinline__ int cmp_batch(const uint8_t* tokens, int64_t a, int64_t b, uint64_t b0,
                                         const RowFmt& f) {
    const uint8_t* ra = row_of(tokens, a, f);
    const uint64_t a0 = pack_word(ra, 0, f);
    if (a0 != b0) return a0 < b0 ? -1 : 1;
    const uint8_t* rb = row_of(tokens, b, f);
    for (int w = 1; w < f.W; ++w) {
        const uint64_t x = pack_word(ra, w, f), y = pack_word(rb, w, f);
        if (x != y) return x < y ? -1 : 1;
    }
    return 0;
}

// Old sorted row p <= batch row j (word 0 = b0)?  Equal old rows have smaller
// ids, so they precede the new row.
__device__ __forceinline__ bool old_le(const uint64_t* __restrict__ rows, const uint64_t* __restrict__ head,
                                       int64_t p, const uint8_t* rj, uint64_t b0, const RowFmt& f) {
    const uint64_t h = head[p];
    if (h != b0) return h < b0;
    for (int w = 1; w < f.W; ++w) {
        const uint64_t x = rows[p * f.W + w], y = pack_word(rj, w, f);
        if (x != y) return x < y;
    }
    return true;
}

// Small batches, one warp per batch row j (batch order):
//   rank  = #{batch rows ordered before j (row, then batch index)},
//   below = #{old rows <= row j} by a 33-way search over the old rows,
// then the row lands in sorted slot `rank` with id N + j and merged output
// position below + rank.  Replaces a separate pack / rank / scatter / locate.
__global__ void __launch_bounds__(128) k_ins_place(const uint8_t* __restrict__ tokens, RowFmt f, int64_t n,
                                                   const uint64_t* __restrict__ old_rows,
                                                   const uint64_t* __restrict__ old_head, int64_t N,
                                                   uint64_t* __restrict__ srows, int32_t* __restrict__ sids,
                                                   int64_t* __restrict__ np) {
    const int64_t j = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
    if (j >= n) return;
    const unsigned lane = lane_id();
    const uint8_t* rj = row_of(tokens, j, f);
    const uint64_t b0 = pack_word(rj, 0, f);
    int rank = 0;
    for (int64_t r0 = 0; r0 < n; r0 += 32) {
        const int64_t r = r0 + lane;
        bool before = false;
        if (r < n && r != j) {
            const int c = cmp_batch(tokens, r, j, b0, f);
            before = c < 0 || (c == 0 && r < j);
        }
        rank += __popc(__ballot_sync(0xffffffffu, before));
    }
    // the old rows satisfying old_le form a prefix: shrink [lo, hi] around
    // its end with 32 probes per round
    int64_t lo = 0, hi = N;
    while (hi - lo > 32) {
        const int64_t p = lo + ((hi - lo) * (int64_t)(lane + 1)) / 33;
        const bool t = old_le(old_rows, old_head, p, rj, b0, f);
        const int c = __popc(__ballot_sync(0xffffffffu, t));
        const int64_t plast = __shfl_sync(0xffffffffu, p, c > 0 ? c - 1 : 0);
        const int64_t pnext = __shfl_sync(0xffffffffu, p, c < 32 ? c : 31);
        if (c > 0) lo = plast + 1;
        if (c < 32) hi = pnext;
    }
    const bool t = lo + (int64_t)lane < hi && old_le(old_rows, old_head, lo + lane, rj, b0, f);
    const int64_t below = lo + __popc(__ballot_sync(0xffffffffu, t));
    for (int w = (int)lane; w < f.W; w += 32) srows[(int64_t)rank * f.W + w] = pack_word(rj, w, f);
    if (lane == 0) {
        sids[rank] = (int32_t)(N + j);
        np[rank] = below + rank;
    }
}

// Large batches: sorted new rows and ids (id = N + batch index) from the
// packed batch and its sorted order.
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

// Large batches: np[j] = j + #{old rows <= new row j}.
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

constexpr int kMergeRows = 256;  // output rows per merge CTA

struct MergeArgs {
    const uint64_t* old_rows;
    const int32_t* old_ids;
    const uint8_t* old_H;
    const uint64_t* srows;  // sorted new rows
    const int32_t* sids;
    const int64_t* np;      // merged position of each sorted new row (ascending)
    int64_t n, total;
    int W, L, tpw, bits;
    uint64_t* rows;  // merged outputs
    uint64_t* head;
    int32_t* ids;
    uint8_t* H;
    int32_t* pos;
    int32_t* bkt;    // depth-1 buckets, updated in place
    int64_t ntok;
    int old_empty;   // the old bucket table was never written
    unsigned merge_ctas;
};

__device__ __forceinline__ int row_lcp(const uint64_t* a, const uint64_t* b, const MergeArgs& m) {
    for (int w = 0; w < m.W; ++w) {
        const uint64_t x = a[w] ^ b[w];
        if (x) {
            const int l = w * m.tpw + (__clzll((long long)x) / m.bits);
            return l < m.L ? l : m.L;
        }
    }
    return m.L;
}

// Merge-path insertion in one pass (Algorithm 1's output, updated rather
// than rebuilt).  Output slot o holds new row j when np[j] == o, else old row
// o - #{np < o}.  Per slot the CTA also writes ids, pos (the inverse
// permutation) and H: an old row whose predecessor is its old predecessor
// keeps its old H entry, only slots next to a new row compare rows.  CTAs
// past merge_ctas shift the depth-1 bucket table instead:
//   bkt[t] += #{new rows whose first token < t}.
__global__ void __launch_bounds__(kMergeRows) k_ins_merge(MergeArgs m) {
    __shared__ int64_t snp[kMergeRows];
    __shared__ int64_t ssrc[kMergeRows];  // >= 0: old row, < 0: -(sorted new row) - 1
    __shared__ int64_t sj0;
    __shared__ int sprev_new;
    const int tid = threadIdx.x;
    if (blockIdx.x >= m.merge_ctas) {
        const int64_t t = (int64_t)(blockIdx.x - m.merge_ctas) * kMergeRows + tid;
        if (t > m.ntok) return;
        int64_t lo = 0, hi = m.n;  // #{new rows with first token < t}
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)(m.srows[mid * m.W] >> (64 - m.bits)) < t) lo = mid + 1;
            else hi = mid;
        }
        m.bkt[t] = (m.old_empty ? 0 : m.bkt[t]) + (int32_t)lo;
        return;
    }
    const int64_t o0 = (int64_t)blockIdx.x * kMergeRows;
    if (tid == 0) {
        int64_t lo = 0, hi = m.n;  // #{np < o0}
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (m.np[mid] < o0) lo = mid + 1;
            else hi = mid;
        }
        sj0 = lo;
        sprev_new = lo > 0 && m.np[lo - 1] == o0 - 1;
    }
    __syncthreads();
    const int64_t j0 = sj0;
    const int64_t avail = m.n - j0 < kMergeRows ? m.n - j0 : kMergeRows;
    snp[tid] = tid < avail ? m.np[j0 + tid] : INT64_MAX;
    __syncthreads();
    const int64_t o = o0 + tid;
    const int rows_here = (int)(m.total - o0 < kMergeRows ? m.total - o0 : kMergeRows);
    if (o < m.total) {
        int lo = 0, hi = (int)avail;  // local #{np < o}
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (snp[mid] < o) lo = mid + 1;
            else hi = mid;
        }
        const int64_t j = j0 + lo;
        const bool is_new = lo < avail && snp[lo] == o;
        // slot o - 1 is new: a new row of this CTA's range, or (first slot only)
        // the last new row before the range
        const bool prev_new = lo > 0 ? snp[lo - 1] == o - 1 : (tid == 0 && sprev_new);
        const int64_t i = o - j;  // old row index when !is_new
        const int32_t id = is_new ? m.sids[j] : m.old_ids[i];
        m.ids[o] = id;
        m.pos[id] = (int32_t)o;
        uint8_t h = 0;
        if (o > 0) {
            if (!is_new && !prev_new) {
                h = m.old_H[i];
            } else {
                const uint64_t* cur = is_new ? m.srows + j * m.W : m.old_rows + i * m.W;
                const uint64_t* prv = prev_new ? m.srows + (j - 1) * m.W : m.old_rows + (o - 1 - j) * m.W;
                h = (uint8_t)row_lcp(prv, cur, m);
            }
        }
        m.H[o] = h;
        ssrc[tid] = is_new ? -(j + 1) : i;
    }
    __syncthreads();
    // rows and head, one thread per output word
    const int W = m.W;
    for (int e = tid; e < rows_here * W; e += kMergeRows) {
        const int r = e / W, w = e - r * W;
        const int64_t src = ssrc[r];
        const uint64_t v = src >= 0 ? m.old_rows[src * W + w] : m.srows[(-src - 1) * W + w];
        m.rows[(o0 + r) * W + w] = v;
        if (w == 0) m.head[o0 + r] = v;
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
    uint64_t* srows = x->ins_rows;
    int32_t* sids = x->ins_ids;
    int64_t* np = x->ins_rank;
    uint64_t* packed = nullptr;
    int32_t* order = nullptr;
    const bool own = !small;
    lcp_buffers& ob = x->buf[x->cur];
    lcp_buffers& nb = x->buf[1 - x->cur];
    int rc = LCP_OK;
    if (small) {
        LCP_TIMED_LAUNCH(k_ins_place, nblocks(n, 4), 128, 0, s, reinterpret_cast<const uint8_t*>(d_tokens), f, n,
                   ob.rows, ob.head, x->N, srows, sids, np);
    } else {
        LCP_CUDA_TRY(cudaMallocAsync((void**)&srows, sizeof(uint64_t) * n * W, s));
        LCP_CUDA_TRY(cudaMallocAsync((void**)&sids, sizeof(int32_t) * n, s));
        LCP_CUDA_TRY(cudaMallocAsync((void**)&np, sizeof(int64_t) * n, s));
        LCP_CUDA_TRY(cudaMallocAsync((void**)&order, sizeof(int32_t) * n, s));
        LCP_CUDA_TRY(cudaMallocAsync((void**)&packed, sizeof(uint64_t) * n * W, s));
        LCP_TIMED_LAUNCH(k_ins_pack, nblocks(n * W, 256), 256, 0, s, reinterpret_cast<const uint8_t*>(d_tokens),
                   f, n, W, packed);
        rc = build_sorted_ids(d_tokens, f, n, order, x->status, s);
        if (rc == LCP_OK) {
            LCP_TIMED_LAUNCH(k_ins_sorted, nblocks(n * W, 256), 256, 0, s, packed, order, n, W, x->N, srows,
                       sids);
            LCP_TIMED_LAUNCH(k_ins_locate, nblocks(n, 128), 128, 0, s, ob.rows, ob.head, x->N, srows, n, W, np);
        }
    }
    if (rc == LCP_OK) {
        MergeArgs m;
        m.old_rows = ob.rows;
        m.old_ids = ob.ids;
        m.old_H = ob.H;
        m.srows = srows;
        m.sids = sids;
        m.np = np;
        m.n = n;
        m.total = x->N + n;
        m.W = W;
        m.L = x->L;
        m.tpw = x->tpw;
        m.bits = x->bits;
        m.rows = nb.rows;
        m.head = nb.head;
        m.ids = nb.ids;
        m.H = nb.H;
        m.pos = x->pos;
        m.bkt = x->bkt;
        m.ntok = 1ll << x->bits;
        m.old_empty = x->N == 0;
        m.merge_ctas = nblocks(m.total, kMergeRows);
        LCP_TIMED_LAUNCH(k_ins_merge, m.merge_ctas + nblocks(m.ntok + 1, kMergeRows), kMergeRows, 0, s, m);
        x->cur = 1 - x->cur;
        x->N = m.total;
        rc = build_aux(x, s, /*merged=*/true);
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
