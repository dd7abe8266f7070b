// Declarations of the full-scan kernels defined in scan.cu, for callers in
// other translation units that supply their own scratch memory.
#pragma once

#include "common.cuh"

namespace lcpk {

// Log entries per (slice, query) beyond k in k_scan_partial: the log is
// compacted back to k entries at most every kLogSlack rows it takes.
constexpr int kLogSlack = 64;

// Threads per CTA of k_scan_partial (its launch bound; a CTA owns that many
// queries of one N-slice, a warp 32 neighbouring ones in the batch order).
constexpr int kScanPartialThreads = 256;

// Keys one k_scan_merge CTA sorts in shared memory at a time, and the most
// N-slices (lists per query) it takes.
constexpr int kMergeCap = 4096;
constexpr int kMergeMaxLists = 2048;

// Largest batch ordered by one CTA (k_query_sort_cta); larger batches take
// the radix sort.
constexpr int kQuerySortCta = 4096;

// The packed first words of the rows, as two arrays -- upper halves, then
// lower halves -- each starting 256-byte aligned and readable up to a
// 16-byte multiple (the bulk copies round their sizes up).
__global__ void k_pack_plane0(const uint8_t* __restrict__ tokens, RowFmt f, int64_t n,
                              uint32_t* __restrict__ plane_hi, uint32_t* __restrict__ plane_lo);

struct ScanArgs {
    const uint8_t* tokens;    // [N, L] raw rows
    const uint32_t* plane_hi;  // packed word 0 of every row: upper halves
    const uint32_t* plane_lo;  // and lower halves
    RowFmt f;
    int64_t N;                // rows scanned: [0, N), in slices of `slice`
    const uint8_t* queries;   // [Q, L] raw queries
    RowFmt qf;
    int64_t Q;
    const int32_t* order;     // batch position -> query (null: identity)
    int32_t* floor;           // per batch position: a level with k rows at or above it, read
                              // as the scan goes and raised (atomic maximum) by every slice
                              // that finds one (null: none; else zeroed before the first pass)
    int k, cap;               // cap = k + kLogSlack entries per log
    int64_t slice;
    uint64_t* lists;          // [S][Q][cap]: each (slice, position) leaves its candidates first
    int32_t* counts;          // [S][Q]: how many (<= k) | the slice's known level << 16 (null: not written)
    int* status;              // device status word (a bounded wait that ran out), may be null
};

// Plane words per slice are a multiple of this (the slices' first words stay
// 16-byte aligned for the bulk copies of the plane tiles).
constexpr int64_t kScanSliceAlign = 64;

// grid = (ceil(Q / kScanPartialThreads), S slices), slices of a multiple
// of kScanSliceAlign rows (the last may be shorter).
__global__ void k_scan_partial(const ScanArgs a);

// grid = Q (batch positions): the k best of each position's S lists into the
// query's output row.  Dynamic shared memory: kMergeCap keys.
__global__ void k_scan_merge(const uint64_t* __restrict__ lists, const int32_t* __restrict__ counts, int cap,
                             int64_t Q, int S, int k, const int32_t* __restrict__ order,
                             int32_t* __restrict__ out_ids, uint8_t* __restrict__ out_lcp);

}  // namespace lcpk

namespace lcph {

// Batches up to this size take the threshold selection (scan_select.cu),
// larger ones the per-thread logs (scan.cu).
constexpr int64_t kSelMaxQ = 1024;

// Full scan of a batch of at most kSelMaxQ queries by threshold selection.
int scan_select(const void* d_tokens, int64_t N, const lcpk::RowFmt& f, const void* d_queries,
                const lcpk::RowFmt& qf, int64_t Q, int k, int32_t* d_out_ids, uint8_t* d_out_lcp, cudaStream_t s);

}  // namespace lcph
