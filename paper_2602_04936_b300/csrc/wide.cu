// Top-1 retrieval with 16-bit LCPs, for rows of up to LCP_MAX_L_WIDE tokens:
// the paper's sustained benchmark (Sec. 7, Table 4; the sustained-load
// configuration of App. C) answers one query at a time with the single best
// item over 2M sequences of max_len 256, whose LCP with a query reaches 256
// and so needs more than 8 bits.
//
// The indexed top-1 needs no adjacent-LCP array.  With p the insertion point
// of q among the sorted rows, d = max(LCP(q, row p-1), LCP(q, row p)) is the
// largest LCP of q with any row (Algorithm 3's descent depth: LCP with a
// fixed string is unimodal over sorted rows), the rows with LCP >= d are the
// contiguous interval of rows sharing q's first d tokens (the descent lemma,
// App. A: items outside T_v have LCP < d), and the answer is its smallest id
// (Definition "Top-k LCP Retrieval" with k = 1: ties broken by index).  One
// warp per query:
//   1. p: binary search inside q's first-token bucket, on the rows' first
//      words (head) and then, among rows with q's first word, on whole rows;
//   2. the LCPs with rows p-1 and p, d their maximum;
//   3. the interval's ends: binary searches for the first and last rows of
//      the bucket whose first d tokens equal q's (a prefix compare per probe);
//   4. its smallest id: two partial 128-row blocks (sorted ids with offsets)
//      and at most two sparse-table lists, whose first entries are the
//      minima of their blocks.
// The full scan computes the LCP of q with every row and keeps the smallest
// key (0xFFFF - LCP) << 32 | id: a per-block minimum, then one 64-bit atomic
// minimum per block and query (order independent, so deterministic).
#include "search.cuh"

namespace lcpk {

constexpr int kWideWarps = 4;
constexpr int kMaxWideW = (LCP_MAX_L_WIDE + 3) / 4;  // packed words of the longest uint16 row
constexpr unsigned kFull = 0xffffffffu;

// True when the first d tokens of sorted row p equal q's (d >= 1).
__device__ __forceinline__ bool warp_prefix_eq(const DevIndex& ix, int64_t p, const uint64_t* q, int d) {
    const unsigned lane = lane_id();
    const int full = d / ix.tpw;        // whole words that must be equal
    const int rem = d - full * ix.tpw;  // leading tokens of word `full` that must be equal
    const int nw = full + (rem ? 1 : 0);
    const uint64_t* row = ix.rows + p * ix.W;
    for (int w0 = 0; w0 < nw; w0 += 32) {
        const int w = w0 + (int)lane;
        bool ne = false;
        if (w < nw) {
            uint64_t x = row[w] ^ q[w];
            if (w == full) x &= ~0ull << (64 - rem * ix.bits);  // here 0 < rem < tpw
            ne = x != 0;
        }
        if (__any_sync(kFull, ne)) return false;
    }
    return true;
}

// First position x in [lo, hi) with head[x] > v (gt) or >= v (!gt).
__device__ __forceinline__ int64_t head_bound(const uint64_t* __restrict__ head, int64_t lo, int64_t hi,
                                              uint64_t v, bool gt) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const uint64_t h = head[mid];
        if (gt ? h <= v : h < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Smallest id at sorted positions [lo, hi) (lo < hi), from the sorted
// 128-position blocks and the sparse table of their smallest ids.
__device__ __forceinline__ uint32_t warp_min_id(const DevIndex& ix, int64_t lo, int64_t hi) {
    const unsigned lane = lane_id();
    const int64_t bl0 = lo / kBlk, bh0 = (hi - 1) / kBlk;
    int64_t pb[2] = {-1, -1};
    int o1[2] = {0, 0}, o2[2] = {0, 0};
    int64_t full_lo = 0, full_hi = 0;  // whole blocks [full_lo, full_hi)
    if (bl0 == bh0) {
        pb[0] = bl0;
        o1[0] = (int)(lo - bl0 * kBlk);
        o2[0] = (int)(hi - bl0 * kBlk);
    } else {
        full_lo = bl0;
        full_hi = bh0 + 1;
        if (lo % kBlk) {
            pb[0] = bl0;
            o1[0] = (int)(lo % kBlk);
            o2[0] = kBlk;
            full_lo = bl0 + 1;
        }
        if (hi != ix.N && (hi % kBlk)) {
            pb[1] = bh0;
            o1[1] = 0;
            o2[1] = (int)(hi % kBlk);
            full_hi = bh0;
        }
    }
    uint32_t best = kInf;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        if (pb[s] < 0) continue;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int t = (int)lane + 32 * e;
            const uint32_t id = ix.sblk[pb[s] * kBlk + t];
            const int off = ix.soff[pb[s] * kBlk + t];
            if (id != kInf && off >= o1[s] && off < o2[s]) best = min(best, id);
        }
    }
    if (full_hi > full_lo && lane == 0) {
        const int64_t span = full_hi - full_lo;
        const int j = 63 - __clzll((long long)span);
        if (j == 0) {
            best = min(best, ix.sblk[full_lo * kBlk]);
        } else {
            const uint32_t* lev = ix.st + (size_t)(j - 1) * (size_t)ix.st_stride * (size_t)ix.K;
            best = min(best, lev[(size_t)full_lo * ix.K]);
            best = min(best, lev[(size_t)(full_hi - (1ll << j)) * ix.K]);
        }
    }
    return __reduce_min_sync(kFull, best);
}

__global__ void __launch_bounds__(kWideWarps * 32) k_top1_wide(DevIndex ix, const uint8_t* __restrict__ queries,
                                                               RowFmt qf, int64_t Q, int32_t* __restrict__ out_ids,
                                                               uint16_t* __restrict__ out_lcp) {
    __shared__ uint64_t qs[kWideWarps][kMaxWideW];
    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const int64_t q = (int64_t)blockIdx.x * kWideWarps + warp;
    if (q >= Q) return;  // warp-uniform
    uint64_t* qw = qs[warp];
    const uint8_t* qrow = row_of(queries, q, qf);
    for (int w = (int)lane; w < ix.W; w += 32) qw[w] = pack_word(qrow, w, qf);
    __syncwarp();
    if (ix.N == 0) {
        if (lane == 0) {
            out_ids[q] = -1;
            out_lcp[q] = 0;
        }
        return;
    }
    // 1. insertion point inside the first-token bucket
    const uint64_t q0 = qw[0];
    const int64_t t0 = (int64_t)(q0 >> (64 - ix.bits));
    const int64_t blo = ix.bkt[t0], bhi = ix.bkt[t0 + 1];
    const int64_t a = head_bound(ix.head, blo, bhi, q0, false);
    const int64_t b = head_bound(ix.head, a, bhi, q0, true);
    int64_t lo = a, hi = b;  // rows [a, b) share q's first word: compare whole rows
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        int l;
        if (warp_cmp_row(ix.rows + mid * ix.W, qw, ix, &l) < 0) lo = mid + 1;
        else hi = mid;
    }
    const int64_t p = lo;
    // 2. the descent depth d
    int lL, lR;
    warp_lcp_neighbours(ix, p, qw, &lL, &lR);
    const int d = max(lL, lR);
    uint32_t id = 0;  // d == 0: no row shares q's first token, every row ties at 0
    if (d > 0) {
        // 3. rows sharing q's first d tokens: [first, last], inside the bucket
        int64_t first = p, last = p - 1;
        if (lL == d) {
            int64_t l0 = blo, h0 = p - 1;  // row p-1 qualifies
            while (l0 < h0) {
                const int64_t mid = (l0 + h0) >> 1;
                if (warp_prefix_eq(ix, mid, qw, d)) h0 = mid;
                else l0 = mid + 1;
            }
            first = l0;
        }
        if (lR == d) {
            int64_t l0 = p + 1, h0 = bhi;  // first row after p that does not qualify
            while (l0 < h0) {
                const int64_t mid = (l0 + h0) >> 1;
                if (warp_prefix_eq(ix, mid, qw, d)) l0 = mid + 1;
                else h0 = mid;
            }
            last = l0 - 1;
        }
        // 4. its smallest id
        id = warp_min_id(ix, first, last + 1);
        if (id == kInf) flag_status(ix.status, DEV_BAD);
    }
    if (lane == 0) {
        out_ids[q] = (int32_t)id;
        out_lcp[q] = (uint16_t)d;
    }
}

// ---- full scan ----

constexpr int kWideScanThreads = 256;

__global__ void __launch_bounds__(kWideScanThreads) k_scan_top1_wide(const uint8_t* __restrict__ tokens, RowFmt f,
                                                                     int64_t N, const uint8_t* __restrict__ queries,
                                                                     RowFmt qf, int64_t slice,
                                                                     unsigned long long* __restrict__ best) {
    __shared__ uint64_t qw[kMaxWideW];
    __shared__ unsigned long long wmin[kWideScanThreads / 32];
    const int64_t q = blockIdx.y;
    const uint8_t* qrow = row_of(queries, q, qf);
    for (int w = threadIdx.x; w < f.W; w += blockDim.x) qw[w] = pack_word(qrow, w, qf);
    __syncthreads();
    const int64_t s0 = (int64_t)blockIdx.x * slice;
    const int64_t s1 = s0 + slice < N ? s0 + slice : N;
    unsigned long long m = ~0ull;
    for (int64_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
        const uint8_t* row = row_of(tokens, i, f);
        int l = f.L;
        for (int w = 0; w < f.W; ++w) {
            const uint64_t x = pack_word(row, w, f) ^ qw[w];
            if (x) {
                l = lcp_at(w, x, f);
                break;
            }
        }
        const unsigned long long key = ((unsigned long long)(0xFFFF - l) << 32) | (unsigned long long)i;
        m = key < m ? key : m;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(kFull, m, o);
        m = y < m ? y : m;
    }
    if (lane_id() == 0) wmin[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kWideScanThreads / 32; ++w) m = wmin[w] < m ? wmin[w] : m;
        if (m != ~0ull) atomicMin(best + q, m);
    }
}

__global__ void k_scan_top1_wide_out(const unsigned long long* __restrict__ best, int64_t Q,
                                     int32_t* __restrict__ out_ids, uint16_t* __restrict__ out_lcp) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    const unsigned long long k = best[q];
    out_ids[q] = (int32_t)(uint32_t)k;
    out_lcp[q] = (uint16_t)(0xFFFF - (int)(k >> 32));
}

}  // namespace lcpk

using namespace lcph;

extern "C" int lcp_top1_wide(lcp_index_t x, const void* d_queries, int64_t Q, int32_t* d_out_ids,
                             uint16_t* d_out_lcp, lcp_stream_t stream) {
    using namespace lcpk;
    if (!x || Q < 0) return LCP_ERR_INVALID;
    if (Q == 0) return LCP_OK;
    if (!d_queries || !d_out_ids || !d_out_lcp) return LCP_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const DevIndex ix = dev_view(x);
    const RowFmt qf = make_fmt(x->tb, x->L, d_queries);
    LCP_TIMED_LAUNCH(k_top1_wide, (unsigned)((Q + kWideWarps - 1) / kWideWarps), kWideWarps * 32, 0, s, ix,
                     reinterpret_cast<const uint8_t*>(d_queries), qf, Q, d_out_ids, d_out_lcp);
    note_use(x, s);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LCP_OK : cuda_status(e);
}

extern "C" int lcp_scan_top1_wide(const void* d_tokens, int64_t N, lcp_format_t fmt, const void* d_queries,
                                  int64_t Q, int32_t* d_out_ids, uint16_t* d_out_lcp, lcp_stream_t stream) {
    using namespace lcpk;
    if ((fmt.token_bytes != 1 && fmt.token_bytes != 2) || fmt.L < 1 || fmt.L > LCP_MAX_L_WIDE || N < 0 ||
        N >= (1ll << 30) || Q < 0)
        return LCP_ERR_INVALID;
    if (Q == 0) return LCP_OK;
    if (!d_queries || !d_out_ids || !d_out_lcp || (N > 0 && !d_tokens)) return LCP_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    if (N == 0) {
        LCP_CUDA_TRY(cudaMemsetAsync(d_out_ids, 0xFF, sizeof(int32_t) * (size_t)Q, s));
        LCP_CUDA_TRY(cudaMemsetAsync(d_out_lcp, 0, sizeof(uint16_t) * (size_t)Q, s));
        return LCP_OK;
    }
    const RowFmt f = make_fmt(fmt.token_bytes, fmt.L, d_tokens);
    const RowFmt qf = make_fmt(fmt.token_bytes, fmt.L, d_queries);
    // about four CTAs per SM over all (slice, query) pairs, slices of >= 4,096 rows
    int64_t S = ((int64_t)sm_count() * 4 + Q - 1) / Q;
    const int64_t maxS = (N + 4095) / 4096;
    if (S > maxS) S = maxS;
    if (S > 65535) S = 65535;
    if (S < 1) S = 1;
    const int64_t slice = (N + S - 1) / S;
    S = (N + slice - 1) / slice;
    unsigned long long* best = nullptr;
    LCP_CUDA_TRY(cudaMallocAsync((void**)&best, sizeof(unsigned long long) * (size_t)Q, s));
    cudaError_t e = cudaMemsetAsync(best, 0xFF, sizeof(unsigned long long) * (size_t)Q, s);
    const uint8_t* qb = reinterpret_cast<const uint8_t*>(d_queries);
    for (int64_t q0 = 0; e == cudaSuccess && q0 < Q; q0 += 65535) {  // grid.y holds the query
        const int64_t qn = Q - q0 < 65535 ? Q - q0 : 65535;
        LCP_TIMED_LAUNCH(k_scan_top1_wide, dim3((unsigned)S, (unsigned)qn), kWideScanThreads, 0, s,
                         reinterpret_cast<const uint8_t*>(d_tokens), f, N, qb + (size_t)q0 * f.row_bytes, qf,
                         slice, best + q0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        LCP_TIMED_LAUNCH(k_scan_top1_wide_out, (unsigned)((Q + 255) / 256), 256, 0, s, best, Q, d_out_ids, d_out_lcp);
        e = cudaGetLastError();
    }
    cudaFreeAsync(best, s);
    return e == cudaSuccess ? LCP_OK : cuda_status(e);
}
