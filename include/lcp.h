/*
 * lcp.h -- C ABI of the B300 library for deterministic top-k retrieval under
 * Longest-Common-Prefix similarity.
 *
 * Problem (paper Sec. 2.1, Definitions "LCP Similarity" and "Top-k LCP
 * Retrieval"): a set S = {s_1..s_N} of sequences of L tokens, a query q and
 * k >= 1 (Algorithm 3 requires an integer k >= 1).  LCP(s, t) is the length
 * of the longest common prefix.  The answer is the k items with the highest
 * LCP(q, s_i), ties broken by original index, so that a fixed (S, q, k)
 * always yields bit-identical output (Theorem 7, "Determinism").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Ids are 0-based original indices: item s_{i+1} of the paper has id i.
 *    Ties are broken by ascending id.  Rows appended by lcp_index_insert take
 *    ids N, N+1, ... in batch row order.
 *  - Tokens are unsigned integers of `token_bytes` (1 = uint8, 2 = uint16)
 *    stored row-major, contiguous, [n, L].  Order is unsigned lexicographic.
 *    1 <= L <= 255 so that an LCP fits in one byte.
 *  - Results are [Q, k] row-major: out_ids (int32) and out_lcp (uint8).  Row r
 *    lists query r's answer in order (LCP descending, id ascending).  When
 *    k > N the slots from N on hold id -1 and lcp 0.
 *  - Pointers named d_* are device pointers (cudaMalloc / torch CUDA memory)
 *    on the current device; h_* are host pointers (pinned memory gives the
 *    fastest copies, pageable memory works).  The caller owns every token,
 *    query and output buffer and must keep it valid until the work enqueued on
 *    `stream` has completed.  The library owns index memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are stream-ordered and asynchronous unless stated.
 *  - Argument errors are returned synchronously and nothing is enqueued.
 *    Errors that arise on the device (a bounded wait that ran out) are
 *    recorded in a device status word and reported by lcp_index_sync /
 *    lcp_device_status; no kernel of this library traps or spins forever.
 *  - Every entry point returns LCP_OK (0) or a negative LCP_ERR_* code;
 *    lcp_status_string gives its text.
 *  - Limits: N <= 2^30 - 1 items per index, k <= LCP_SCAN_MAX_K for the full
 *    scan and k <= the index's max_k (<= LCP_INDEX_MAX_K) for indexed search.
 *  - Rows longer than 255 tokens (up to LCP_MAX_L_WIDE) are served top-1
 *    only, with 16-bit LCPs: lcp_top1_wide / lcp_scan_top1_wide below.
 */
#ifndef LCP_H_
#define LCP_H_

#include <stdint.h>

#if defined(__GNUC__)
#define LCP_API __attribute__((visibility("default")))
#else
#define LCP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define LCP_OK 0
#define LCP_PENDING 1           /* session ticket not finished yet */
#define LCP_ERR_INVALID (-1)    /* bad argument: null pointer, k < 1, L out of range ... */
#define LCP_ERR_OOM (-2)        /* device allocation failed */
#define LCP_ERR_CAPACITY (-3)   /* insert would exceed the index capacity */
#define LCP_ERR_BUDGET (-4)     /* request can never fit the session memory budget */
#define LCP_ERR_TIMEOUT (-5)    /* a bounded device or host wait ran out */
#define LCP_ERR_CUDA (-6)       /* a CUDA runtime call failed */
#define LCP_ERR_STATE (-7)      /* object in the wrong state (destroyed, shut down) */

#define LCP_INDEX_MAX_K 128     /* largest max_k an index can be built for */
#define LCP_SCAN_MAX_K 1024     /* largest k for lcp_scan_topk */
#define LCP_MAX_L 255
#define LCP_MAX_L_WIDE 1024     /* longest rows of a top-1 ("wide") index */

typedef void* lcp_stream_t; /* a cudaStream_t */
typedef struct lcp_index_s* lcp_index_t;

/* Token format of a dataset: 1 or 2 bytes per token, L tokens per row.
 * vocab is informational (0 = unknown); tokens are not range-checked. */
typedef struct {
    int32_t token_bytes;
    int32_t L;
    int32_t vocab;
} lcp_format_t;

LCP_API const char* lcp_status_string(int status);

/* ------------------------------------------------------------------------
 * Index build -- Algorithm 1 (BuildLCPIndex, Sec. 5.2) and Algorithm 2
 * (subtree sizes) in array form.
 *
 * Builds the prefix index of the N rows at d_tokens ([N, L], device memory):
 * the rows packed into 64-bit words and sorted lexicographically (equal rows
 * by id), their ids in that order, the adjacent-LCP array H (H[p] =
 * LCP(row p-1, row p)), and the auxiliary tables the search uses to break
 * ties by index.  The trie's nodes are the LCP intervals of H; a node's
 * subtree size |T_v| is its interval length.
 *   capacity: rows the index can hold without reallocating (>= N; 0 = N).
 *             lcp_index_insert fails with LCP_ERR_CAPACITY beyond it.
 *   max_k:    largest k lcp_topk_batch will accept (1..LCP_INDEX_MAX_K).
 * fmt.L may exceed LCP_MAX_L (up to LCP_MAX_L_WIDE) only with max_k = 1 and
 * capacity = N: such a "wide" index is answered by lcp_top1_wide alone (the
 * 8-bit-LCP calls -- lcp_topk_batch, insert, BFS, TAL, the session, the
 * queue, graph steps, the tuner and the export of H -- return
 * LCP_ERR_INVALID for it).
 * On success *out owns the device memory; release it with lcp_index_destroy.
 * The build runs as one CUDA graph on `stream` and the call blocks the host
 * until the device has finished its sort (an event recorded mid-graph): the
 * host then reads how many rows sit in tie groups too large for the
 * on-device group sort (more than 2,048 rows sharing packed word 0, or a
 * group of 33 to 2,048 in which a row shares word 1 with more than 64
 * others).  Usually none do and the call returns while the device finishes
 * the build's second half; otherwise those rows are ordered exactly by
 * host-driven refinement rounds (more waits).  Inside a stream capture the
 * build runs as plain launches with the same waits.  d_tokens may be reused
 * once the stream has passed the build.
 * Errors: LCP_ERR_INVALID, LCP_ERR_OOM, LCP_ERR_CUDA.
 * ---------------------------------------------------------------------- */
LCP_API int lcp_index_build(const void* d_tokens, int64_t N, lcp_format_t fmt, int64_t capacity,
                    int32_t max_k, lcp_stream_t stream, lcp_index_t* out);

/* Same, with the tokens in host memory; the host-to-device copy is part of
 * the call, enqueued on `stream` before the build.  From pinned memory the
 * copy is asynchronous: keep h_tokens unchanged until the stream has passed
 * it (lcp_index_sync or a stream synchronise); pageable memory is copied
 * before the call returns.  The call's input copy follows this thread's
 * earlier host-buffer input copies on the link (see lcp_topk_batch_host). */
LCP_API int lcp_index_build_host(const void* h_tokens, int64_t N, lcp_format_t fmt, int64_t capacity,
                         int32_t max_k, lcp_stream_t stream, lcp_index_t* out);

/* ------------------------------------------------------------------------
 * Insert -- dynamic updates (the paper's static analysis leaves them to
 * future work, Sec. 10.1 / App. G).  Appends n rows ([n, L], device memory,
 * same format) with ids N..N+n-1: the batch is sorted, merged into the sorted
 * rows by merge path (on equal rows the older, smaller id first), and H and
 * the tie tables are refreshed.  The result is byte-identical to building the
 * concatenated dataset from scratch.  Never reallocates; fails with
 * LCP_ERR_CAPACITY if N + n > capacity.  Batches of up to
 * LCP_INSERT_SMALL_BATCH rows never block the host; larger batches may
 * (like lcp_index_build).
 * ---------------------------------------------------------------------- */
#define LCP_INSERT_SMALL_BATCH 2048
LCP_API int lcp_index_insert(lcp_index_t index, const void* d_tokens, int64_t n, lcp_stream_t stream);

/* ------------------------------------------------------------------------
 * Indexed batched top-k -- Algorithm 3 (descent) with the collection of
 * Algorithm 4 / CollectTopKOptimized (App. D), in the order of the
 * Definition "Top-k LCP Retrieval":
 *   1. binary search for q's insertion point p in the sorted rows and the
 *      LCPs with both neighbours (the descent depth is their maximum);
 *   2. expansion outward from p through H, level by level, until the level
 *      d* at which at least k items have LCP >= d* (all items with LCP > d*
 *      are taken: fewer than k);
 *   3. the remaining slots are filled from the LCP-interval of level d*
 *      (prefix bucket B_{q[1..d*]}, Sec. 6.2) with its smallest ids.
 * d_queries: [Q, L] device memory in the index's format.  1 <= k <= max_k.
 * Output [Q, k] as described above.  Q = 0 is a no-op.
 * ---------------------------------------------------------------------- */
LCP_API int lcp_topk_batch(lcp_index_t index, const void* d_queries, int64_t Q, int32_t k,
                   int32_t* d_out_ids, uint8_t* d_out_lcp, lcp_stream_t stream);

/* Same, with host queries and host outputs; the copies in both directions
 * are part of the call, which returns when the results are in host memory.
 * Large batches are copied, searched and copied back in chunks on two copy
 * streams beside `stream`.  The device staging for queries and results, the
 * copy streams and their events are kept per calling thread and device and
 * reused by later calls (the staging grows to the largest batch and is not
 * released).  A call's query copies wait only for this thread's previous
 * host-buffer input copies (not for the whole of `stream`), so they can
 * overlap a build enqueued just before. */
LCP_API int lcp_topk_batch_host(lcp_index_t index, const void* h_queries, int64_t Q, int32_t k,
                        int32_t* h_out_ids, uint8_t* h_out_lcp, lcp_stream_t stream);

/* ------------------------------------------------------------------------
 * Full scan top-k -- the index-free baseline ("full scan" of Sec. 7, Table 6):
 * LCP of every query against all N rows, keeping per query the k best under
 * (LCP descending, id ascending).  Needs no index.
 * d_tokens [N, L], d_queries [Q, L] device memory in format fmt.
 * 1 <= k <= LCP_SCAN_MAX_K.  Batches of up to 1,024 queries take a
 * threshold selection: one read of each row's first 16 bytes counts, per
 * query and 256-row granule, the rows of LCP >= 1..4 and lists the rows
 * sharing the query's first tokens; d* (the k-th largest LCP) follows from
 * the counts, and the answer comes from a list or from a walk of the few
 * granules holding the rows above d* and the first rows at d* by id.
 * Larger batches are ordered by the queries' first words and keep, per
 * thread and N-slice, the rows that can still be in the query's top k (a
 * log of up to k + 64 rows, compacted as it fills), then merge them.
 * Both return the same bytes.  Temporary device memory from the
 * stream-ordered allocator: about N * 8 + Q * (8 * ceil(N / 256) + 65,536
 * + 4 * (L + 3)) bytes for small batches, and
 * N * 8 + Q * (16 + S * ((k + 64) * 8 + 4)) bytes for larger ones (S <=
 * 2048 slices; plus 24 bytes a query past 4,096 queries for the sort).
 * ---------------------------------------------------------------------- */
LCP_API int lcp_scan_topk(const void* d_tokens, int64_t N, lcp_format_t fmt, const void* d_queries,
                  int64_t Q, int32_t k, int32_t* d_out_ids, uint8_t* d_out_lcp,
                  lcp_stream_t stream);

/* ------------------------------------------------------------------------
 * Top-1 with 16-bit LCPs, for rows of up to LCP_MAX_L_WIDE tokens -- the
 * paper's sustained benchmark (Sec. 7, Table 4; its configuration in App. C:
 * top-1 over 2M sequences of max_len 256, one query at a time), whose LCPs
 * reach 256 and do not fit the 8-bit LCP of the calls above.
 *
 * lcp_top1_wide: indexed.  Any index (built with any max_k; a wide index must
 *   have max_k = 1).  For each query: the insertion point p among the sorted
 *   rows (binary search in the query's first-token bucket), the descent
 *   depth d = max(LCP(q, row p-1), LCP(q, row p)) -- the largest LCP of q
 *   with any row (Algorithm 3) --, the interval of rows sharing q's first d
 *   tokens (the descent lemma, App. A), and its smallest id (ties broken by
 *   index, Definition "Top-k LCP Retrieval" with k = 1).
 * lcp_scan_top1_wide: full scan, no index: the LCP of each query with all N
 *   rows and the smallest id at the largest LCP.  1 <= L <= LCP_MAX_L_WIDE.
 * d_queries [Q, L] device memory in the index's (scan: fmt's) format;
 * d_out_ids [Q] int32 and d_out_lcp [Q] uint16: device memory; N = 0 gives
 * (-1, 0).  Stream-ordered; errors as lcp_topk_batch (the full scan takes
 * Q * 8 bytes of stream-ordered scratch).
 * ---------------------------------------------------------------------- */
LCP_API int lcp_top1_wide(lcp_index_t index, const void* d_queries, int64_t Q, int32_t* d_out_ids,
                          uint16_t* d_out_lcp, lcp_stream_t stream);
LCP_API int lcp_scan_top1_wide(const void* d_tokens, int64_t N, lcp_format_t fmt, const void* d_queries,
                               int64_t Q, int32_t* d_out_ids, uint16_t* d_out_lcp, lcp_stream_t stream);

/* ------------------------------------------------------------------------
 * Full scan top-k without any device allocation.  The paper has no
 * counterpart; this is a deployment variant of lcp_scan_topk for callers that
 * cannot allocate device memory when they call in (a real-time control loop
 * that must not block in the allocator, code restricted to start-up
 * allocation, host code inside a stream capture in global mode).  Same
 * arguments and results as lcp_scan_topk.
 *
 * Scratch: a fixed array of LCP_SCAN_NOALLOC_SCRATCH_BYTES inside the
 * library's device image, held by every GPU that loads the library until the
 * process exits.  A call needs 2 * round_up(N * 4, 256) + round_up(Q * 4, 256)
 * + Q * (k + 64) * 8 bytes of it (the rows' first words in two halves, then
 * one N-slice of per-query logs and their counts); larger requests return
 * LCP_ERR_INVALID without enqueuing anything (split the query batch).  The call allocates nothing: no cudaMalloc, cudaFree or
 * allocating library routine.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) -- make that first call
 * before any stream capture.  Every call shares the one array: calls that
 * overlap on the GPU race, so order them (one stream, or events).
 * ---------------------------------------------------------------------- */
#define LCP_SCAN_NOALLOC_SCRATCH_BYTES (32u << 20)
LCP_API int lcp_scan_topk_noalloc(const void* d_tokens, int64_t N, lcp_format_t fmt,
                                  const void* d_queries, int64_t Q, int32_t k, int32_t* d_out_ids,
                                  uint8_t* d_out_lcp, lcp_stream_t stream);

/* ------------------------------------------------------------------------
 * The paper's own query modes (variants; lcp_topk_batch is the Definition).
 *
 * lcp_topk_bfs -- Algorithms 3 + 4 as printed (Sec. 5.3): descend to the
 *   deepest trie node v on q's path (depth d = the largest LCP of q with any
 *   row) and return the first k items of T_v in BFS order -- for rows of one
 *   length L, T_v's items in sorted-row order, equal rows by id -- each with
 *   LCP d, padded with (-1, 0) when |T_v| < k.  Any k >= 1.
 * lcp_tal_topk -- Thermal-Aware Logic (Definition "TAL", Sec. 6.2, and the
 *   TALRangeScan listing, App. D): the bucket is the rows sharing q's first
 *   `depth` tokens (0 <= depth <= L; B = vocab^depth buckets); only the
 *   bucket's rows are scanned, and its top k by (LCP desc, id asc) are
 *   returned, padded when the bucket holds fewer.  1 <= k <= LCP_TAL_MAX_K.
 * Buffers and errors as lcp_topk_batch.
 * ---------------------------------------------------------------------- */
#define LCP_TAL_MAX_K 32
LCP_API int lcp_topk_bfs(lcp_index_t index, const void* d_queries, int64_t Q, int32_t k, int32_t* d_out_ids,
                         uint8_t* d_out_lcp, lcp_stream_t stream);
LCP_API int lcp_tal_topk(lcp_index_t index, const void* d_queries, int64_t Q, int32_t k, int32_t depth,
                         int32_t* d_out_ids, uint8_t* d_out_lcp, lcp_stream_t stream);

/* ------------------------------------------------------------------------
 * Autotuner for the indexed search's launch shape (the paper has no
 * counterpart; the shape never changes a result).  lcp_autotune times every
 * candidate shape -- one fused kernel with a warp per query (the default for
 * batches of up to 4,096 queries), or locate + answer + fill with 1..32
 * queries per warp of the answer kernel and lane- or warp-per-query location,
 * or lane-per-query location that first searches the top levels of the
 * sorted array staged in shared memory -- on the caller's sample batch (device queries, Q >= 1, k <= max_k) with
 * CUDA events on `stream`, synchronously, and installs the fastest for later
 * lcp_topk_batch calls whose index and batch fall in the same class:
 * (floor(log2 N), L, token bytes, floor(log2 Q), k class {1, <=16, <=64,
 * <=128}), process-wide.  lcp_set_search_shape installs a known shape for
 * that class (to reuse a cached tuning run); qpw = 0 there and in the
 * result means the fused kernel.
 * ---------------------------------------------------------------------- */
typedef struct {
    int32_t qpw;          /* queries per warp chosen; 0: the fused kernel */
    int32_t locate_warp;  /* 1: warp per query, 0: lane per query, 2: lane per query over the
                             staged top levels (4,096 sampled heads in shared memory) */
    float best_ms;        /* its time on the sample batch */
    float default_ms;     /* the untuned heuristic's time */
} lcp_tune_result_t;
LCP_API int lcp_autotune(lcp_index_t index, const void* d_queries, int64_t Q, int32_t k, lcp_stream_t stream,
                         lcp_tune_result_t* best);
LCP_API int lcp_set_search_shape(lcp_index_t index, int64_t Q, int32_t k, int32_t qpw, int32_t locate_warp);

/* ------------------------------------------------------------------------
 * Persistent search fed by a device work queue (the batched serving path:
 * requests against several resident indexes of uneven N, L and k run in one
 * long-lived launch instead of a launch per request).  The paper runs one
 * query stream per process; the queue is this library's.
 *
 * Each request is cut into tasks of whole queries; its records are copied
 * to a device-memory task ring and the new task count after them, on one
 * copy stream.  Warps of the persistent kernel claim tasks (compare-and-swap
 * on a device counter), answer them exactly as lcp_topk_batch does, and
 * publish the request's ticket to mapped host memory.
 * Warps that find no work for idle_ms exit; a later submit or poll relaunches
 * the kernel.  Every device wait is bounded.
 *
 * Queries and outputs are device memory and must stay valid until the
 * ticket completes; the queries must be fully written (their producing
 * stream synchronized) before submit, since the running kernel cannot wait
 * on a stream.  The index must not change (insert) while requests against
 * it are in flight.  Submit returns LCP_ERR_CAPACITY when max_requests
 * requests or max_tasks tasks are in flight: poll and retry.  Poll returns
 * LCP_OK once the request is complete, LCP_PENDING at the timeout.
 * Destroy waits for outstanding requests, then stops the worker.
 * ---------------------------------------------------------------------- */
typedef struct lcp_queue_s* lcp_queue_t;
typedef struct {
    int32_t max_requests;  /* in flight at once (1 .. 65536) */
    int32_t max_tasks;     /* task ring entries (1 .. 2^24) */
    double idle_ms;        /* a warp with no work for this long exits (> 0) */
    int32_t ctas_per_sm;   /* worker CTAs per SM (1 .. 32) */
} lcp_queue_cfg_t;
LCP_API int lcp_queue_create(const lcp_queue_cfg_t* cfg, lcp_queue_t* out);
LCP_API int lcp_queue_submit(lcp_queue_t q, lcp_index_t index, const void* d_queries, int64_t Q, int32_t k,
                             int32_t* d_out_ids, uint8_t* d_out_lcp, uint64_t* ticket);
LCP_API int lcp_queue_poll(lcp_queue_t q, uint64_t ticket, int32_t timeout_ms);
LCP_API int lcp_queue_stats(lcp_queue_t q, int64_t* inflight, int64_t* worker_launches);
LCP_API int lcp_queue_destroy(lcp_queue_t q);
/* Open-loop replay: request i is submitted at arrival_s[i] seconds after the
 * call starts (later if the queue is full: arrival order is kept); its
 * latency, completion time minus arrival time in seconds, lands in
 * latency_s[i] (-1 if rejected or unfinished at timeout_s); *wall_s = time of
 * the last completion.  Device buffers as for lcp_queue_submit. */
typedef struct {
    double arrival_s;
    lcp_index_t index;
    int32_t k;
    int64_t Q;
    const void* d_queries;
    int32_t* d_out_ids;
    uint8_t* d_out_lcp;
} lcp_queue_replay_req_t;
LCP_API int lcp_queue_replay(lcp_queue_t q, const lcp_queue_replay_req_t* reqs, int64_t n, double timeout_s,
                             double* latency_s, double* wall_s);

/* ------------------------------------------------------------------------
 * Sharded index: merge of per-shard answers.  The rows are partitioned by
 * original-id range over P shards (shard s holds global ids h_bases[s] ..),
 * each shard's index answers the same Q queries with its local ids, and this
 * call merges the P answers into the global top k.  Each shard row is ordered
 * by (LCP desc, id asc) as lcp_topk_batch returns it, so the global answer is
 * the k smallest keys (255 - lcp) << 32 | (base + id) over all shards -- the
 * same bytes a single index over all rows returns (Definition "Top-k LCP
 * Retrieval"; keys are unique).  The paper runs one index; the sharded
 * layout is this library's.
 * d_ids [P, Q, k] int32 and d_lcp [P, Q, k] uint8: device, shard-major, as
 * P stacked lcp_topk_batch outputs (padding id -1 allowed); h_bases [P]: host,
 * 0 <= base < 2^31; d_out_* [Q, k]: device.  1 <= P <= LCP_SHARD_MAX.
 * ---------------------------------------------------------------------- */
#define LCP_SHARD_MAX 32
LCP_API int lcp_shard_merge(const int32_t* d_ids, const uint8_t* d_lcp, int32_t P, const int64_t* h_bases,
                            int64_t Q, int32_t k, int32_t* d_out_ids, uint8_t* d_out_lcp, lcp_stream_t stream);

/* ------------------------------------------------------------------------
 * Streaming step as a CUDA graph: insert n rows, then answer Q queries --
 * the guidance/navigation stream of the paper (Sec. 1 Example 1, Sec. 7
 * Table 7: every control step stores the current sensor readings and
 * queries them).  Each run captures the step's kernels on a private stream
 * (nothing executes during capture), updates the instantiated graph in place
 * (cudaGraphExecUpdate) and launches it on `stream`, so the whole step runs
 * without per-kernel launch gaps.  When the update is refused -- the number
 * of kernels changed because N grew past a level boundary of the min tree
 * or sparse table -- the graph is instantiated anew.
 * Requires n <= LCP_INSERT_SMALL_BATCH (the insert path that never waits for
 * the device), room for the rows (else LCP_ERR_CAPACITY), 1 <= k <= max_k.
 * d_insert [n, L], d_queries [Q, L], d_out_* [Q, k]: device memory.  The step
 * owns its scratch; the index must outlive it.
 * ---------------------------------------------------------------------- */
typedef struct lcp_step_s* lcp_step_t;
LCP_API int lcp_step_create(lcp_index_t index, int64_t n, int64_t Q, int32_t k, lcp_step_t* out);
LCP_API int lcp_step_run(lcp_step_t step, const void* d_insert, const void* d_queries, int32_t* d_out_ids,
                         uint8_t* d_out_lcp, lcp_stream_t stream);
/* Runs so far and how many of them had to instantiate the graph anew. */
LCP_API int lcp_step_stats(lcp_step_t step, int64_t* runs, int64_t* instantiations);
LCP_API int lcp_step_destroy(lcp_step_t step);

/* ------------------------------------------------------------------------
 * Serving session -- continuous batching over resident indexes.  Not in the
 * paper (its sustained benchmark, Sec. 7 Table 4, serves one query at a
 * time); this is the serving layer around lcp_topk_batch.
 *
 * A session holds several built indexes (lcp_session_add_index; the caller
 * keeps ownership and must not destroy them before the session).  Each
 * submitted request (queries [Q, L] in the index's format, k, outputs
 * [Q, k]; each buffer in host or device memory -- the session copies with
 * unified addressing, so either works) counts Q*(L*token_bytes + 16 + 5*k)
 * bytes against the budget while in flight.  The session allocates mem_budget (+ 1 KB) of
 * device memory once, in lcp_session_create (LCP_ERR_OOM if that fails), and
 * carves each request's query, id and LCP buffers from it: no request
 * allocates device memory (lcp_topk_batch of more than 4,096 queries still
 * takes its search scratch from the stream-ordered pool).  The memory is
 * freed by lcp_session_destroy.  Requests are admitted in arrival order while at most
 * max_inflight are on the GPU and their memory fits mem_budget; the rest wait
 * and are admitted as earlier requests complete, so requests that arrive
 * while others run join them on the GPU (spread over `streams` CUDA streams,
 * where their copies and kernels overlap).  A request whose memory alone
 * exceeds mem_budget is rejected with LCP_ERR_BUDGET.  Each result is
 * exactly what lcp_topk_batch returns for that request alone.
 * Query and output buffers must stay valid (and device queries fully
 * written) until the request's ticket completes; pinned host memory makes
 * host copies asynchronous.
 * All calls are thread-safe.  dry_run = 1 runs the admission logic without a
 * device (requests complete on the next poll), for testing the policy.
 * ---------------------------------------------------------------------- */
typedef struct lcp_session_s* lcp_session_t;
typedef struct {
    int64_t mem_budget;    /* device bytes for requests in flight (> 0) */
    int32_t max_inflight;  /* requests on the GPU at once (>= 1) */
    int32_t streams;       /* CUDA streams (1..64) */
    int32_t dry_run;       /* 1: no device work (policy tests) */
} lcp_session_cfg_t;
typedef struct {
    int64_t submitted, admitted, completed, rejected;
    int64_t inflight, pending;
    int64_t mem_in_use, mem_peak;
} lcp_session_stats_t;

LCP_API int lcp_session_create(const lcp_session_cfg_t* cfg, lcp_session_t* out);
/* Registers an index; *slot receives its number (0, 1, ...). */
LCP_API int lcp_session_add_index(lcp_session_t session, lcp_index_t index, int32_t* slot);
/* Registers a resident token set ([N, L] device memory in format fmt, kept
 * valid and unchanged by the caller for the session's life) answered by the
 * full scan (lcp_scan_topk), so that the index-free baseline is served the
 * same way as an index; k <= LCP_SCAN_MAX_K.  A request counts
 * Q*(L*token_bytes + 5*k) bytes against the budget (its queries and
 * results, carved from the session's memory); the scan's own temporaries
 * come from the stream-ordered pool. */
LCP_API int lcp_session_add_scan(lcp_session_t session, const void* d_tokens, int64_t N, lcp_format_t fmt,
                                 int32_t* slot);
/* Queues a request; *ticket identifies it.  Never blocks on the device.
 * queries, out_ids and out_lcp: host or device pointers (see above). */
LCP_API int lcp_session_submit(lcp_session_t session, int32_t slot, const void* queries, int64_t Q,
                               int32_t k, int32_t* out_ids, uint8_t* out_lcp, uint64_t* ticket);
/* Advances the session (retires finished requests, admits waiting ones) and
 * reports the ticket: LCP_OK when its results are in the host buffers,
 * LCP_PENDING if it is not done within timeout_ms (0 = just check), or the
 * request's error.  A ticket reports LCP_OK once; later polls return
 * LCP_ERR_INVALID. */
LCP_API int lcp_session_poll(lcp_session_t session, uint64_t ticket, int32_t timeout_ms);
LCP_API int lcp_session_stats(lcp_session_t session, lcp_session_stats_t* stats);
/* Waits for requests on the GPU (up to 10 s), cancels waiting ones, frees
 * the session.  Returns LCP_ERR_TIMEOUT if the wait ran out. */
LCP_API int lcp_session_destroy(lcp_session_t session);

/* Open-loop load driver: submits reqs[i] when its arrival time (seconds from
 * the call's start, non-decreasing) comes, polls completions, and writes
 * latency_s[i] = completion time - scheduled arrival time (so a driver that
 * falls behind is charged for it); a rejected request gets -1.  *wall_s is
 * the time from the first arrival to the last completion.  Blocks until
 * every request is done or timeout_s passes (LCP_ERR_TIMEOUT). */
typedef struct {
    double arrival_s;
    int32_t slot;
    int32_t k;
    int64_t Q;
    const void* h_queries;
    int32_t* h_out_ids;
    uint8_t* h_out_lcp;
} lcp_replay_req_t;
LCP_API int lcp_session_replay(lcp_session_t session, const lcp_replay_req_t* reqs, int64_t n,
                               double timeout_s, double* latency_s, double* wall_s);

/* ------------------------------------------------------------------------
 * Index inspection and lifetime.
 * ---------------------------------------------------------------------- */
/* Current item count and device bytes held (both may be NULL). Synchronous,
 * host-side only. */
LCP_API int lcp_index_size(lcp_index_t index, int64_t* N, int64_t* bytes);

/* Copies the sorted order (ids, [N] int32) and the adjacent-LCP array (H,
 * [N] uint8) of the index to device buffers; either may be NULL.  For tests
 * and checkpoints. */
LCP_API int lcp_index_export(lcp_index_t index, int32_t* d_ids, uint8_t* d_H, lcp_stream_t stream);

/* Waits for the index's most recent operation (on whichever stream it was
 * issued; the index records an event of its own after each call) and
 * reports any device status (LCP_ERR_TIMEOUT if a bounded device wait ran
 * out), then clears it. */
LCP_API int lcp_index_sync(lcp_index_t index);

/* Frees the index.  It may have been used on several streams, some perhaps
 * destroyed since, so this waits for the whole device first.  NULL is a
 * no-op. */
LCP_API int lcp_index_destroy(lcp_index_t index);

/* ------------------------------------------------------------------------
 * Library-wide diagnostics.
 * ---------------------------------------------------------------------- */
/* Synchronises the device and reports, then clears, the library's device
 * status word (written by kernels that are not tied to an index). */
LCP_API int lcp_device_status(void);

/* Number of kernels this library has launched in this process. */
LCP_API int64_t lcp_launch_count(void);

/* Per-kernel timing for profiling (the paper has no counterpart).  While
 * enabled, the search, scan and insert kernels are bracketed by CUDA events
 * on their launching stream (not inside a stream capture); enabling clears
 * the accumulated figures.  lcp_kernel_time waits for the recorded events
 * and returns the total device time and launch count of the kernels whose
 * name starts with `prefix` (e.g. "k_topk_answer").  Adds two event records
 * per launch, so leave it off where launch overhead matters. */
LCP_API int lcp_kernel_timing(int enable);
/* How lcp_index_build issues its kernels (process-wide; profiling aid, the
 * paper has no counterpart): enable = 1 (the default) replays them as one
 * CUDA graph; 0 launches them directly on the build's streams, so that
 * lcp_kernel_timing can bracket each build kernel (a graph's launches
 * carry no events).  The index built is the same either way.  Returns
 * LCP_OK. */
LCP_API int lcp_build_graph(int enable);
/* Restricts the timing to kernels whose name starts with `prefix` (NULL or
 * "" = every timed kernel), so that timing a few kernels adds no event
 * records to the others. */
LCP_API int lcp_kernel_timing_filter(const char* prefix);
LCP_API int lcp_kernel_time(const char* prefix, double* total_ms, int64_t* launches);

/* Test hook for the bounded-wait machinery: launches one kernel that waits
 * for a device flag nobody sets, with the given spin limit, and returns the
 * status that kernel reports (LCP_ERR_TIMEOUT when the limit is reached).
 * Never traps and never hangs. */
LCP_API int lcp_debug_bounded_wait(int64_t spin_limit, lcp_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* LCP_H_ */
