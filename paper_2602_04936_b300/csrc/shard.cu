// Merge of per-shard top-k lists (the sharded layout of the index: the rows
// are partitioned by original-id range, every shard answers the same queries
// against its own index, and the shard answers are merged).
//
// Each shard's row of k results is ordered by the key (255 - lcp) << 32 | id
// -- the order of the Definition "Top-k LCP Retrieval" -- and stays ordered
// when its local ids are shifted by the shard's first global id.  The global
// top k is therefore the k smallest keys over all shards' lists: a k-way
// merge.  Keys are unique (global ids differ), so the result does not depend
// on the merge order and equals the single-index answer bit for bit.
#include "index.cuh"

namespace lcpk {

struct ShardBases {
    int64_t base[LCP_SHARD_MAX];
};

__device__ __forceinline__ uint64_t shard_key(const int32_t* ids, const uint8_t* lcp, int64_t at,
                                              int64_t base) {
    const int32_t id = ids[at];
    if (id < 0) return ~0ull;  // padding: the shard had fewer than k rows
    return ((uint64_t)(255u - lcp[at]) << 32) | (uint64_t)(base + id);
}

// One warp per query; lane s < P holds the head of shard s's list.  Each of
// the k rounds takes the warp minimum (a butterfly of 64-bit shuffles) and
// advances the lane that held it.
__global__ void __launch_bounds__(256) k_shard_merge(const int32_t* __restrict__ ids, const uint8_t* __restrict__ lcp,
                                                     int P, int64_t Q, int k, ShardBases bases,
                                                     int32_t* __restrict__ out_ids, uint8_t* __restrict__ out_lcp) {
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= Q) return;
    const int lane = (int)lane_id();
    const bool mine = lane < P;
    const int64_t row = mine ? ((int64_t)lane * Q + q) * k : 0;
    int head = 0;
    uint64_t key = mine ? shard_key(ids, lcp, row, bases.base[lane]) : ~0ull;
    for (int r = 0; r < k; ++r) {
        uint64_t m = key;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const uint64_t y = __shfl_xor_sync(0xffffffffu, m, o);
            m = y < m ? y : m;
        }
        if (lane == 0) {
            out_ids[q * k + r] = m == ~0ull ? -1 : (int32_t)(m & 0xffffffffu);
            out_lcp[q * k + r] = m == ~0ull ? 0 : (uint8_t)(255u - (uint32_t)(m >> 32));
        }
        if (m != ~0ull && key == m) {  // keys are unique: exactly one lane advances
            ++head;
            key = head < k ? shard_key(ids, lcp, row + head, bases.base[lane]) : ~0ull;
        }
    }
}

}  // namespace lcpk

extern "C" int lcp_shard_merge(const int32_t* d_ids, const uint8_t* d_lcp, int32_t P, const int64_t* h_bases,
                               int64_t Q, int32_t k, int32_t* d_out_ids, uint8_t* d_out_lcp,
                               lcp_stream_t stream) {
    if (P < 1 || P > LCP_SHARD_MAX || Q < 0 || k < 1 || !h_bases) return LCP_ERR_INVALID;
    if (Q > 0 && (!d_ids || !d_lcp || !d_out_ids || !d_out_lcp)) return LCP_ERR_INVALID;
    lcpk::ShardBases b;
    for (int s = 0; s < P; ++s) {
        if (h_bases[s] < 0 || h_bases[s] >= (1ll << 31)) return LCP_ERR_INVALID;
        b.base[s] = h_bases[s];
    }
    if (Q == 0) return LCP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    LCP_LAUNCH(lcpk::k_shard_merge, (unsigned)((Q + 7) / 8), 256, 0, s, d_ids, d_lcp, P, Q, k, b, d_out_ids,
               d_out_lcp);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LCP_OK : lcph::cuda_status(e);
}
