// The paper's own query modes, beside the Definition-order search:
//
//  * BFS order (Algorithms 3 + 4 as printed): descend to the deepest node v
//    on q's path and return the first k items of T_v in BFS order.  Rows all
//    have length L, so items sit at depth-L leaves only, BFS meets them in
//    lexicographic order and equal rows in id order: T_v is the level-d
//    interval of the sorted array around q (d = max LCP) and the answer is
//    its first k positions, each with LCP d.  One warp per query: locate,
//    close the interval on the min tree, copy ids.
//  * TAL (Definition "TAL" and TALRangeScan, Sec. 6.2 / App. D): the bucket
//    of q's d-symbol prefix is found, then only the bucket's rows are
//    scanned -- LCP computed from the packed words of every row, no use of
//    H -- and its top k by (LCP desc, id asc) returned.  One CTA per query
//    (per query and part of its bucket for small batches, the parts' lists
//    merged afterwards); each warp keeps a sorted list of its k best keys
//    (lane j holds the j-th smallest (255 - lcp) << 32 | id) and inserts the
//    rare candidates below its k-th key; warp 0 merges the eight lists.
#include "search.cuh"

namespace lcpk {

// Level-d interval around insertion point p: rows whose first d tokens equal
// q's.  lL, lR = LCP of q with rows p-1, p (-1 where absent).  Empty (lo ==
// hi == p) when neither neighbour reaches d.
__device__ __forceinline__ void level_interval(const DevIndex& ix, int64_t p, int lL, int lR, int d,
                                               int64_t* lo, int64_t* hi) {
    if (d <= 0) {
        *lo = 0;
        *hi = ix.N;
        return;
    }
    const bool inL = lL >= d, inR = lR >= d;
    int xl = -1, xr = (int)ix.N;
    if (inL || inR) find_bounds(ix, (int)p - 1, inL, (int)p + 1, inR, d, &xl, &xr);
    *lo = inL ? (xl < 0 ? 0 : xl) : p;
    *hi = inR ? xr : p;
}

__global__ void __launch_bounds__(256) k_bfs_answer(DevIndex ix, const QLoc* __restrict__ loc, int64_t Q, int k,
                                                    int32_t* __restrict__ out_ids, uint8_t* __restrict__ out_lcp) {
    const int64_t qi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (qi >= Q) return;
    const unsigned lane = lane_id();
    const QLoc r = loc[qi];
    const int d = r.lL > r.lR ? r.lL : r.lR;  // descent depth (N >= 1: one neighbour exists)
    int64_t lo, hi;
    level_interval(ix, r.p, r.lL, r.lR, d, &lo, &hi);
    const int64_t n = hi - lo < k ? hi - lo : k;
    for (int t = (int)lane; t < k; t += 32) {
        out_ids[qi * k + t] = t < n ? ix.ids[lo + t] : -1;
        out_lcp[qi * k + t] = t < n ? (uint8_t)d : 0;
    }
}

constexpr int kTalWarps = 8;

// Inserts candidate key c into the warp's ascending list (lane j = j-th
// smallest, lanes >= k hold ~0): lanes at or past its rank shift up by one.
__device__ __forceinline__ uint64_t list_insert(uint64_t list, uint64_t c, unsigned lane) {
    const int pos = __popc(__ballot_sync(0xffffffffu, list < c));
    const uint64_t up = __shfl_up_sync(0xffffffffu, list, 1);
    return (int)lane < pos ? list : ((int)lane == pos ? c : up);
}

__global__ void __launch_bounds__(kTalWarps * 32) k_tal_scan(DevIndex ix, const uint8_t* __restrict__ queries,
                                                             RowFmt qf, const QLoc* __restrict__ loc, int64_t Q,
                                                             int k, int depth, int32_t* __restrict__ out_ids,
                                                             uint8_t* __restrict__ out_lcp) {
    __shared__ uint64_t qw[kMaxW];
    __shared__ uint64_t lists[kTalWarps][32];
    __shared__ int64_t bounds[2];
    const int64_t qi = blockIdx.x;
    const int part = blockIdx.y, parts = gridDim.y;  // the bucket is split over `parts` CTAs
    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const uint8_t* qrow = row_of(queries, qi, qf);
    for (int w = threadIdx.x; w < ix.W; w += blockDim.x) qw[w] = pack_word(qrow, w, qf);
    if (warp == 0) {
        const QLoc r = loc[qi];
        int64_t lo, hi;
        level_interval(ix, r.p, r.lL, r.lR, depth, &lo, &hi);
        if (lane == 0) {
            bounds[0] = lo;
            bounds[1] = hi;
        }
    }
    __syncthreads();
    const int64_t lo = bounds[0], hi = bounds[1];
    uint64_t list = ~0ull;
    uint64_t thr = ~0ull;  // the list's k-th key
    for (int64_t b = lo + ((int64_t)part * kTalWarps + warp) * 32; b < hi; b += (int64_t)parts * kTalWarps * 32) {
        const int64_t x = b + lane;
        uint64_t key = ~0ull;
        if (x < hi) {
            const uint64_t* row = ix.rows + x * ix.W;
            int l = ix.L;
            for (int w = 0; w < ix.W; ++w) {
                const uint64_t v = row[w] ^ qw[w];
                if (v) {
                    l = w * ix.tpw + (__clzll((long long)v) / ix.bits);
                    l = l < ix.L ? l : ix.L;
                    break;
                }
            }
            key = ((uint64_t)(255 - l) << 32) | (uint32_t)ix.ids[x];
        }
        unsigned m = __ballot_sync(0xffffffffu, key < thr);
        while (m) {
            const int src = __ffs(m) - 1;
            list = list_insert(list, __shfl_sync(0xffffffffu, key, src), lane);
            thr = __shfl_sync(0xffffffffu, list, k - 1);
            m &= ~(1u << src);
            m &= __ballot_sync(0xffffffffu, key < thr);
        }
    }
    lists[warp][lane] = list;
    __syncthreads();
    if (warp != 0) return;
    for (int w = 1; w < kTalWarps; ++w) {
        const uint64_t other = lists[w][lane];
        unsigned m = __ballot_sync(0xffffffffu, (int)lane < k && other < thr);
        while (m) {
            const int src = __ffs(m) - 1;
            list = list_insert(list, __shfl_sync(0xffffffffu, other, src), lane);
            thr = __shfl_sync(0xffffffffu, list, k - 1);
            m &= ~(1u << src);
            m &= __ballot_sync(0xffffffffu, (int)lane < k && other < thr);
        }
    }
    if ((int)lane < k) {  // part-major [parts, Q, k] when the bucket is split
        const int64_t o = ((int64_t)part * Q + qi) * k + lane;
        out_ids[o] = list == ~0ull ? -1 : (int32_t)(list & 0xffffffffu);
        out_lcp[o] = list == ~0ull ? 0 : (uint8_t)(255u - (uint32_t)(list >> 32));
    }
}

}  // namespace lcpk

namespace lcph {
using namespace lcpk;

enum class Mode { kBfs, kTal };

static int run_mode(lcp_index_s* x, const void* d_queries, int64_t Q, int k, int depth, int32_t* out_ids,
                    uint8_t* out_lcp, cudaStream_t s, Mode mode) {
    if (Q <= 0) return LCP_OK;
    if (x->N == 0) {
        LCP_CUDA_TRY(cudaMemsetAsync(out_ids, 0xFF, sizeof(int32_t) * (size_t)Q * k, s));
        LCP_CUDA_TRY(cudaMemsetAsync(out_lcp, 0, (size_t)Q * k, s));
        return LCP_OK;
    }
    DevIndex ix = dev_view(x);
    RowFmt qf = make_fmt(x->tb, x->L, d_queries);
    const uint8_t* q = reinterpret_cast<const uint8_t*>(d_queries);
    QLoc* loc = nullptr;
    LCP_CUDA_TRY(cudaMallocAsync((void**)&loc, sizeof(QLoc) * (size_t)Q, s));
    launch_locate(ix, q, qf, Q, loc, s);
    if (mode == Mode::kBfs) {
        LCP_TIMED_LAUNCH(k_bfs_answer, (unsigned)((Q + 7) / 8), 256, 0, s, ix, loc, Q, k, out_ids, out_lcp);
    } else {
        // small batches split each bucket over several CTAs (two waves of the
        // GPU in total), whose partial top-k lists are then merged
        int parts = (int)((2 * (int64_t)sm_count() + Q - 1) / Q);
        parts = parts < 1 ? 1 : (parts > LCP_SHARD_MAX ? LCP_SHARD_MAX : parts);
        int32_t* pid = out_ids;
        uint8_t* plcp = out_lcp;
        if (parts > 1) {
            LCP_CUDA_TRY(cudaMallocAsync((void**)&pid, sizeof(int32_t) * (size_t)parts * Q * k, s));
            LCP_CUDA_TRY(cudaMallocAsync((void**)&plcp, (size_t)parts * Q * k, s));
        }
        LCP_TIMED_LAUNCH(k_tal_scan, dim3((unsigned)Q, (unsigned)parts), kTalWarps * 32, 0, s, ix, q, qf, loc, Q, k,
                         depth, pid, plcp);
        if (parts > 1) {
            const int64_t zero[LCP_SHARD_MAX] = {0};  // part lists already hold global ids
            const int rc = lcp_shard_merge(pid, plcp, parts, zero, Q, k, out_ids, out_lcp, s);
            cudaFreeAsync(pid, s);
            cudaFreeAsync(plcp, s);
            if (rc != LCP_OK) return rc;
        }
    }
    LCP_CUDA_TRY(cudaFreeAsync(loc, s));
    return LCP_OK;
}

}  // namespace lcph

extern "C" {

int lcp_topk_bfs(lcp_index_t x, const void* d_queries, int64_t Q, int32_t k, int32_t* d_out_ids,
                 uint8_t* d_out_lcp, lcp_stream_t stream) {
    if (!x || Q < 0 || k < 1 || lcph::index_is_wide(x)) return LCP_ERR_INVALID;
    if (Q > 0 && (!d_queries || !d_out_ids || !d_out_lcp)) return LCP_ERR_INVALID;
    int rc = lcph::run_mode(x, d_queries, Q, k, 0, d_out_ids, d_out_lcp, (cudaStream_t)stream, lcph::Mode::kBfs);
    if (rc == LCP_OK) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = lcph::cuda_status(e);
    }
    lcph::note_use(x, (cudaStream_t)stream);
    return rc;
}

int lcp_tal_topk(lcp_index_t x, const void* d_queries, int64_t Q, int32_t k, int32_t depth, int32_t* d_out_ids,
                 uint8_t* d_out_lcp, lcp_stream_t stream) {
    if (!x || Q < 0 || k < 1 || k > LCP_TAL_MAX_K || depth < 0 || depth > x->L || lcph::index_is_wide(x))
        return LCP_ERR_INVALID;
    if (Q > 0 && (!d_queries || !d_out_ids || !d_out_lcp)) return LCP_ERR_INVALID;
    int rc = lcph::run_mode(x, d_queries, Q, k, depth, d_out_ids, d_out_lcp, (cudaStream_t)stream,
                            lcph::Mode::kTal);
    if (rc == LCP_OK) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = lcph::cuda_status(e);
    }
    lcph::note_use(x, (cudaStream_t)stream);
    return rc;
}

}  // extern "C"
