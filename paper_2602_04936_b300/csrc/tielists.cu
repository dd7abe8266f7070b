// Tie lists of heavy trie nodes (the augmentation of Sec. 5.1: each node of
// the trie also carries, here, the K smallest ids in its subtree).
//
// The trie's nodes are the LCP intervals of H.  Every interval of more than
// 128 rows contains a sample position 128*s.  For each sample, one warp walks
// its chain of heavy ancestors from the root down: at depth d the interval
// around the sample is closed with the min tree, its LCP value l (the minimum
// H inside it) says that depths d..l give the same interval, and the walk
// continues at depth l + 1 until the interval holds 128 rows or fewer.  The
// interval is recorded under (first sample inside it, l), a key unique per
// trie node; the sample whose index is that first sample marks it canonical.
// A scan numbers the canonical nodes (deterministically, in key order), one
// warp per node takes its K smallest ids from the sparse table, and the
// per-sample table is rewritten from node keys to list numbers.  Nodes beyond
// the list capacity keep -1 and the search falls back to the sparse table.
// Nothing here reads back to the host, so inserts stay graph-capturable.
#include "search.cuh"

namespace lcpk {

constexpr int kTlWarps = 4;
constexpr int kScanBlk = 2048;  // flags per scan block (256 threads x 8)

__global__ void __launch_bounds__(kTlWarps * 32) k_heavy_intervals(DevIndex ix, int64_t nsamp,
                                                                   int32_t* __restrict__ tbl,
                                                                   uint8_t* __restrict__ flag,
                                                                   int32_t* __restrict__ slo,
                                                                   int32_t* __restrict__ shi) {
    const int64_t i = ((int64_t)blockIdx.x * kTlWarps + (threadIdx.x >> 5));
    if (i >= nsamp) return;
    const unsigned lane = lane_id();
    const int64_t s = i * kBlk;
    const int L1 = ix.L1, L = ix.L1 - 1;
    int d = 0;
    int64_t lo = 0, hi = ix.N;
    for (;;) {
        if (hi - lo <= kBlk) break;
        int ell = range_min_H(ix, lo + 1, hi - 1);
        if (ell > L) ell = L;
        if (ell < d) ell = d;  // cannot happen: every H inside is >= d
        const int64_t c = (lo + kBlk - 1) / kBlk;
        const int64_t slot = c * L1 + ell;
        for (int dd = d + (int)lane; dd <= ell; dd += 32) tbl[i * L1 + dd] = (int32_t)slot;
        if (c == i && lane == 0) {
            flag[slot] = 1;
            slo[slot] = (int32_t)lo;
            shi[slot] = (int32_t)hi;
        }
        d = ell + 1;
        if (d > L) break;
        int xl, xr;
        find_bounds(ix, (int)s, true, (int)s + 1, true, d, &xl, &xr);
        lo = xl < 0 ? 0 : xl;
        hi = xr;
    }
}

// Clears the per-sample node table and the canonical-node flags (one kernel
// rather than two memsets, so a captured graph keeps its node types).
__global__ void k_tl_reset(int32_t* __restrict__ tbl, uint8_t* __restrict__ flag, int64_t n) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    tbl[e] = -1;
    flag[e] = 0;
}

__global__ void __launch_bounds__(256) k_flag_count(const uint8_t* __restrict__ flag, int64_t n,
                                                    uint64_t* __restrict__ sums) {
    __shared__ uint32_t ws[8];
    uint32_t c = 0;
    const int64_t b0 = (int64_t)blockIdx.x * kScanBlk;
    for (int j = 0; j < kScanBlk / 256; ++j) {
        const int64_t e = b0 + j * 256 + threadIdx.x;
        if (e < n) c += flag[e];
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane_id() == 0) ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < 8; ++w) t += ws[w];
        sums[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) k_flag_scan_sums(uint64_t* sums, int64_t nb, uint32_t* total) {
    __shared__ uint64_t tmp[32];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < nb; b0 += 1024) {
        const int64_t i = b0 + threadIdx.x;
        const uint64_t v = i < nb ? sums[i] : 0ull;
        uint64_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane_id() >= (unsigned)o) x += y;
        }
        if (lane_id() == 31) tmp[threadIdx.x >> 5] = x;
        __syncthreads();
        uint64_t add = carry;
        for (unsigned w = 0; w < (threadIdx.x >> 5); ++w) add += tmp[w];
        if (i < nb) sums[i] = add + x - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = add + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = (uint32_t)carry;
}

__global__ void __launch_bounds__(256) k_flag_assign(const uint8_t* __restrict__ flag, int64_t n,
                                                     const uint64_t* __restrict__ offs,
                                                     const int32_t* __restrict__ slo,
                                                     const int32_t* __restrict__ shi, int64_t cap,
                                                     int32_t* __restrict__ slot_list,
                                                     int32_t* __restrict__ tl_lo,
                                                     int32_t* __restrict__ tl_hi) {
    __shared__ uint32_t ws[8];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = offs[blockIdx.x];
    __syncthreads();
    const int64_t b0 = (int64_t)blockIdx.x * kScanBlk;
    for (int j = 0; j < kScanBlk / 256; ++j) {
        const int64_t e = b0 + j * 256 + threadIdx.x;
        const uint32_t f = e < n ? flag[e] : 0u;
        uint32_t x = f;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane_id() >= (unsigned)o) x += y;
        }
        if (lane_id() == 31) ws[threadIdx.x >> 5] = x;
        __syncthreads();
        uint64_t add = carry;
        for (unsigned w = 0; w < (threadIdx.x >> 5); ++w) add += ws[w];
        if (f) {
            const int64_t r = (int64_t)(add + x - f);
            slot_list[e] = r < cap ? (int32_t)r : -1;
            if (r < cap) {
                tl_lo[r] = slo[e];
                tl_hi[r] = shi[e];
            }
        }
        __syncthreads();
        if (threadIdx.x == 255) carry = add + x;
        __syncthreads();
    }
}

// One warp per list: the K smallest ids of the node's interval.
__global__ void __launch_bounds__(kTlWarps * 32) k_node_lists(DevIndex ix, const uint32_t* __restrict__ total,
                                                              int64_t cap, const int32_t* __restrict__ tl_lo,
                                                              const int32_t* __restrict__ tl_hi,
                                                              uint32_t* __restrict__ lists,
                                                              int32_t* __restrict__ lpos) {
    __shared__ QWarp sm[kTlWarps];
    const int64_t w = (int64_t)blockIdx.x * kTlWarps + (threadIdx.x >> 5);
    const int64_t m = *total < (uint64_t)cap ? (int64_t)*total : cap;
    if (w >= m) return;
    QWarp& S = sm[threadIdx.x >> 5];
    const int cm = smallest_ids(ix, tl_lo[w], tl_hi[w], ix.K, S);
    for (int t = (int)lane_id(); t < ix.K; t += 32) {
        const uint32_t id = t < cm ? S.src[0][t] : kInf;
        lists[w * ix.K + t] = id;
        lpos[w * ix.K + t] = id != kInf ? ix.pos[id] : -1;
    }
}

// List of each depth-1 bucket (its interval at depth 1), -1 if light.
__global__ void k_bucket_lists(DevIndex ix, int64_t ntok, int32_t* __restrict__ bkt_list) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntok) return;
    const int64_t lo = ix.bkt[t], hi = ix.bkt[t + 1];
    int32_t li = -1;
    if (hi - lo > kBlk) li = ix.tbl[((lo + kBlk - 1) / kBlk) * ix.L1 + 1];
    bkt_list[t] = li;
}

__global__ void k_remap_tbl(int32_t* __restrict__ tbl, int64_t n, const int32_t* __restrict__ slot_list) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int32_t v = tbl[e];
    if (v >= 0) tbl[e] = slot_list[v];
}

}  // namespace lcpk

namespace lcph {
using namespace lcpk;

int build_tie_lists_nodes(lcp_index_s* x, cudaStream_t s) {
    const int64_t N = x->N;
    if (N <= 0 || !x->tbl) return LCP_OK;
    const int64_t nsamp = (N + kBlk - 1) / kBlk;
    const int L1 = x->L + 1;
    const int64_t nslots = nsamp * L1;
    LCP_TIMED_LAUNCH(k_tl_reset, (unsigned)((nslots + 255) / 256), 256, 0, s, x->tbl, x->slot_flag, nslots);
    DevIndex ix = dev_view(x);
    LCP_TIMED_LAUNCH(k_heavy_intervals, (unsigned)((nsamp + kTlWarps - 1) / kTlWarps), kTlWarps * 32, 0, s, ix,
               nsamp, x->tbl, x->slot_flag, x->slot_lo, x->slot_hi);
    const int64_t nb = (nslots + kScanBlk - 1) / kScanBlk;
    LCP_TIMED_LAUNCH(k_flag_count, (unsigned)nb, 256, 0, s, x->slot_flag, nslots, x->tl_sums);
    LCP_TIMED_LAUNCH(k_flag_scan_sums, 1, 1024, 0, s, x->tl_sums, nb, x->tl_total);
    LCP_TIMED_LAUNCH(k_flag_assign, (unsigned)nb, 256, 0, s, x->slot_flag, nslots, x->tl_sums, x->slot_lo,
               x->slot_hi, x->nlists_cap, x->slot_list, x->tl_lo, x->tl_hi);
    return LCP_OK;
}

int build_tie_lists_fill(lcp_index_s* x, cudaStream_t s) {
    const int64_t N = x->N;
    if (N <= 0 || !x->tbl) return LCP_OK;
    const int64_t nsamp = (N + kBlk - 1) / kBlk;
    const int L1 = x->L + 1;
    const int64_t nslots = nsamp * L1;
    DevIndex ix = dev_view(x);
    LCP_TIMED_LAUNCH(k_node_lists, (unsigned)((x->nlists_cap + kTlWarps - 1) / kTlWarps), kTlWarps * 32, 0, s,
               ix, x->tl_total, x->nlists_cap, x->tl_lo, x->tl_hi, x->tlists, x->tlpos);
    LCP_TIMED_LAUNCH(k_remap_tbl, (unsigned)((nslots + 255) / 256), 256, 0, s, x->tbl, nslots, x->slot_list);
    const int64_t ntok = 1ll << x->bits;
    LCP_TIMED_LAUNCH(k_bucket_lists, (unsigned)((ntok + 255) / 256), 256, 0, s, ix, ntok, x->bkt_list);
    return LCP_OK;
}

}  // namespace lcph
