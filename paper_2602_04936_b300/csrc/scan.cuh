// Declarations of the full-scan kernels defined in scan.cu, for callers in
// other translation units that supply their own scratch memory.
#pragma once

#include "common.cuh"

namespace lcpk {

// Log entries per (slice, query) beyond k in k_scan_partial: the log is
// compacted back to k entries at most every kLogSlack rows it takes.
constexpr int kLogSlack = 64;

// Threads per CTA of k_scan_partial (its launch bound; a CTA owns that many
// queries of one N-slice).
constexpr int kScanPartialThreads = 128;

// Keys one k_scan_merge CTA sorts in shared memory: a merge takes at most
// kMergeCap / (k rounded up to a power of two) lists per query.
constexpr int kMergeCap = 4096;

__global__ void k_pack_plane0(const uint8_t* __restrict__ tokens, RowFmt f, int64_t n,
                              uint64_t* __restrict__ plane0);

// lists: [S][Q][cap] keys, cap = k + kLogSlack; each (slice, query) leaves its
// k best keys (unordered, padded with ~0) in the first k entries of its list.
__global__ void k_scan_partial(const uint8_t* __restrict__ tokens, const uint64_t* __restrict__ plane0,
                               RowFmt f, int64_t N, const uint8_t* __restrict__ queries, RowFmt qf,
                               int64_t Q, int k, int cap, int64_t slice, uint64_t* __restrict__ lists);

__global__ void k_scan_merge(const uint64_t* __restrict__ in, int in_stride, int64_t Q, int k, int nlists,
                             int G, int P, uint64_t* __restrict__ out, int final_pass,
                             int32_t* __restrict__ out_ids, uint8_t* __restrict__ out_lcp);

}  // namespace lcpk
