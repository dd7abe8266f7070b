// Device layout of the prefix index (the array form of the paper's trie).
//
//   rows [cap][W] u64   packed rows in lexicographic order (equal rows by id)
//   head [cap]    u64   word 0 of each sorted row (16 MB at N=2M: L2-resident
//                       for the binary search)
//   ids  [cap]    i32   original id of each sorted row
//   H    [cap]    u8    H[0] = 0, H[p] = LCP(row p-1, row p)   (Alg. 2's subtree
//                       sizes are the lengths of H's LCP intervals)
//   pos  [cap]    i32   inverse of ids (id -> sorted position)
//   hmin          u8    32-ary min tree over H: level j+1 holds the minimum of
//                       32 consecutive level-j entries.  Finds the end of an LCP
//                       interval (next/previous H < d) in a few L2 probes.
//   sblk [nblk][128] u32  ids of each 128-position block sorted ascending
//   soff [nblk][128] u8   the in-block offset of each of those ids
//   st   [lev][nblk][K] u32  sparse table: level j >= 1 at block b holds the K
//                       smallest ids of blocks [b, b + 2^j), ascending; padded
//                       with 0xFFFFFFFF.  Any position range's K smallest ids
//                       come from two partial blocks and two table entries.
//   bkt  [2^bits + 1] i32  depth-1 buckets (TAL's prefix partition with d = 1,
//                       Sec. 6): rows whose first token is t occupy sorted
//                       positions [bkt[t], bkt[t+1]).
//   tbl  [N/128][L+1] i32  tie lists of heavy trie nodes: the LCP interval of
//                       depth d around sample position 128*s, if it holds more
//                       than 128 rows, has its K smallest ids (ascending) in
//                       tlists[tbl[s][d]] and their sorted positions in
//                       tlpos[tbl[s][d]]; -1 otherwise.  Every trie node of
//                       more than 128 rows contains a sample, so the indexed
//                       search finds the level-d* list with one lookup.
//   top  [T]      u64   the top levels of the sorted array for the search:
//                       head at T evenly spaced positions j * N / T, T =
//                       min(N, kTopLevels); staged in shared memory by the
//                       staged locate, which narrows a query's range to about
//                       N / T rows before touching L2.
//   bkt_list [2^bits] i32  the list of each depth-1 bucket (-1 if light), so
//                       that the common d* = 1 case reads bounds and list
//                       number in one round trip.
//   sub  [<=64][2^bits] i32x2  depth-2 buckets (start, end) of depth-1
//                       buckets of at least 4,096 rows: the d* = 2
//                       interval of a query whose first token has a table is
//                       two loads instead of a search (indexes without insert
//                       capacity; sub_idx maps a first token to its table).
#pragma once

#include "common.cuh"

namespace lcpk {

constexpr int kBlk = 128;        // positions per tie-fill block
constexpr int kMaxHLev = 7;      // min-tree levels above H (32^7 > 2^30)
constexpr int kMaxStLev = 24;
constexpr uint32_t kInf = 0xFFFFFFFFu;
constexpr int kTopLevels = 4096;  // samples of the sorted array's heads (32 KB)
constexpr int kSub2Max = 64;       // depth-2 bucket tables at most
constexpr int kSub2Min = 4096;     // rows a depth-1 bucket needs to get one

struct DevIndex {
    int64_t N;
    int W, L, tpw, bits;
    int K;            // tie-list length (multiple of 32, >= max_k)
    int64_t nblk;     // ceil(N / kBlk)
    int hlev;         // number of min-tree levels above H
    int st_levels;    // sparse-table levels stored (1..st_levels)
    const uint64_t* rows;
    const uint64_t* head;
    const int32_t* ids;
    const uint8_t* H;
    const int32_t* pos;
    const uint8_t* hmin;
    int64_t hoff[kMaxHLev + 1];  // offset of level j in hmin (j >= 1)
    int64_t hlen[kMaxHLev + 1];  // entries at level j (hlen[0] = N)
    const uint32_t* sblk;
    const uint8_t* soff;
    const uint32_t* st;
    int64_t st_stride;  // nblk capacity used for the table layout
    const int32_t* bkt;
    // depth-2 buckets of the largest depth-1 buckets (null: none): sub_idx[t0]
    // is t0's table (-1 if none) and sub[(table << bits) + t1] the sorted
    // positions [x, y) of the rows whose first two tokens are (t0, t1), for
    // pairs that occur
    const int32_t* sub_idx;
    const int2* sub;
    const int32_t* tbl;
    const uint32_t* tlists;
    const int32_t* tlpos;
    const int32_t* bkt_list;
    const uint64_t* top;  // [top_n] heads at positions j * N / top_n
    int top_n;
    int L1;  // L + 1: row length of tbl
    int* status;
};

}  // namespace lcpk

struct lcp_buffers {
    uint64_t* rows = nullptr;
    uint64_t* head = nullptr;
    int32_t* ids = nullptr;
    uint8_t* H = nullptr;
};

struct lcp_index_s {
    int device = 0;
    int tb = 0, L = 0, W = 0, tpw = 0, bits = 0, vocab = 0;
    int64_t N = 0, cap = 0;
    int max_k = 0, K = 0;
    lcp_buffers buf[2];
    int cur = 0;
    int32_t* pos = nullptr;
    uint8_t* hmin = nullptr;
    int hlev = 0;
    int64_t hoff[lcpk::kMaxHLev + 1] = {0};
    int64_t hlen[lcpk::kMaxHLev + 1] = {0};
    uint32_t* sblk = nullptr;
    uint8_t* soff = nullptr;
    uint32_t* st = nullptr;
    int32_t* bkt = nullptr;
    // depth-2 bucket tables (indexes without insert capacity only)
    int32_t* sub_idx = nullptr;    // [2^bits]
    int2* sub = nullptr;           // [kSub2Max][2^bits]
    uint32_t* sub_count = nullptr;  // tables handed out
    // heavy-node tie lists
    int32_t* tbl = nullptr;        // [nsamp_cap][L+1]
    uint8_t* slot_flag = nullptr;  // [nsamp_cap][L+1] canonical (sample, depth) slots
    int32_t* slot_lo = nullptr;    // interval of each canonical slot
    int32_t* slot_hi = nullptr;
    int32_t* slot_list = nullptr;  // list index of each canonical slot
    uint32_t* tlists = nullptr;    // [nlists_cap][K]
    int32_t* tlpos = nullptr;      // [nlists_cap][K] sorted position of each entry
    int32_t* bkt_list = nullptr;   // [2^bits] list of each depth-1 bucket
    uint64_t* top = nullptr;       // [kTopLevels] sampled heads (the search's top levels)
    int32_t* tl_lo = nullptr;      // interval of each list
    int32_t* tl_hi = nullptr;
    uint64_t* tl_sums = nullptr;   // scan block sums
    uint32_t* tl_total = nullptr;  // number of canonical slots (device)
    int64_t nsamp_cap = 0, nlists_cap = 0;
    int64_t nblk_cap = 0;
    int st_levels_cap = 0;
    int* status = nullptr;  // device status word
    // streams the index has been used on, each with an event recorded after
    // the last operation there; `shared` once a session or work queue holds
    // it (their streams are not tracked here) or more than kMaxUses streams
    // were seen -- destroy then waits for the whole device
    struct Use {
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
    };
    static constexpr int kMaxUses = 8;
    Use uses[kMaxUses];
    int nuses = 0;
    bool shared = false;
    int64_t bytes = 0;
    void* arena = nullptr;  // one allocation holding every device array above
    // insert scratch (allocated at build when cap > N)
    uint64_t* ins_rows = nullptr;   // [LCP_INSERT_SMALL_BATCH][W] sorted new rows
    int32_t* ins_ids = nullptr;     // ids of the sorted new rows
    int64_t* ins_rank = nullptr;    // output position of each new row
};

namespace lcph {

// An index over rows longer than LCP_MAX_L tokens (built with max_k = 1):
// only lcp_top1_wide answers it; H is clamped to 255 there and unused.
inline bool index_is_wide(const lcp_index_s* x) { return x->L > LCP_MAX_L; }

lcpk::DevIndex dev_view(const lcp_index_s* x);

// Sorts rows of `tokens` and writes their ids in sorted order (build step).
int build_sorted_ids(const void* tokens, const lcpk::RowFmt& f, int64_t N, int32_t* ids_out,
                     int* err, cudaStream_t s, uint32_t* huge_host = nullptr, void* scratch = nullptr);
// Bytes of the scratch block build_sorted_ids takes (instead of allocating).
size_t build_scratch_bytes(int64_t N);
// rows/head/H from raw tokens and sorted ids.
int gather_rows_and_lcp(const void* tokens, const lcpk::RowFmt& f, int64_t N, const int32_t* ids,
                        lcp_buffers& b, int W, cudaStream_t s);
// H from already-packed sorted rows.
int adjacent_lcp(const uint64_t* rows, int64_t N, int W, int L, int tpw, int bits, uint8_t* H,
                 cudaStream_t s);
// pos, min tree and tie tables of the current buffers.
// Records that the index's last operation on stream s was just issued.
void note_use(lcp_index_s* x, cudaStream_t s);

// Rebuilds the derived tables (pos, buckets, min tree, sorted blocks, sparse
// table, tie lists) from the current buffer set; `merged`: an insert's merge
// pass already wrote pos and the buckets.
int build_aux(lcp_index_s* x, cudaStream_t s, bool merged);
// Heavy-node tie lists in two parts: the nodes, their keys and numbering
// (needs the min tree), then their lists and the lookup tables (needs the
// sparse table, pos and the buckets too).
int build_tie_lists_nodes(lcp_index_s* x, cudaStream_t s);
int build_tie_lists_fill(lcp_index_s* x, cudaStream_t s);

// A second stream of this thread for the current device, with a fork and a
// join event: independent branches of the build run on it, ordered against
// the caller's stream by the events only -- concurrent in direct calls,
// parallel branches when captured into a graph.  Created on first use (so
// call it once before any stream capture); nullptr if that failed.
struct SideStream {
    cudaStream_t s2 = nullptr, s3 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, fork3 = nullptr, join3 = nullptr;
};
SideStream* side_stream();

// loc_scratch: caller-owned buffer of search_scratch_bytes(Q) bytes for the
// per-query position records, or nullptr to use stream-ordered scratch.
// Launch shape of the indexed search (see search.cuh).
struct SearchShape {
    int qpw = 32;         // queries per warp of the answer kernel
    int locate_warp = 0;  // 1: warp-per-query locate, 0: lane-per-query
    int fused = 0;        // 1: one kernel, a warp per query (small batches)
};

// The full scan (scan.cu) on stream s: rows [N, L] of tb-byte tokens.
int scan_topk_device(const void* d_tokens, int64_t N, int tb, int L, const void* d_queries, int64_t Q, int k,
                     int32_t* d_out_ids, uint8_t* d_out_lcp, cudaStream_t s);

int topk_batch_device(lcp_index_s* x, const void* d_queries, int64_t Q, int k, int32_t* out_ids,
                      uint8_t* out_lcp, cudaStream_t s, void* loc_scratch = nullptr,
                      const SearchShape* shape = nullptr);
size_t search_scratch_bytes(int64_t Q);
int insert_device(lcp_index_s* x, const void* d_tokens, int64_t n, cudaStream_t s);

}  // namespace lcph
