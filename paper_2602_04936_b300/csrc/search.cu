// Indexed batched top-k (Algorithm 3 + CollectTopK / CollectTopKOptimized,
// returning the order of the Definition "Top-k LCP Retrieval").
//
// Three kernels per large batch, with small per-query records between them
// (one fused kernel stalled on instruction fetch there):
//   locate  the insertion point p of each query (first row >= q) and its
//           LCPs lL, lR with rows p-1 and p, searched inside the depth-1
//           bucket of q's first token: one lane per query over the
//           L2-resident head array (word 0 of every sorted row) for large
//           batches, one warp per query with a 33-way search for small ones.
//           max(lL, lR) is the descent depth of Algorithm 3.
//   answer  one warp per query: expansion -- along each side the LCP of row
//           j with q is the running minimum of H towards p (descent lemma,
//           App. A); 32-item chunks are loaded, 64 per side at once, then
//           from the side whose next LCP is larger, until at least k loaded
//           items have an LCP no smaller than anything not loaded; d* is the
//           k-th largest loaded LCP.  Items with LCP > d* (the set A, fewer
//           than k) are all taken, ordered by (LCP desc, id asc) and written
//           to slots [0, |A|).  The interval [lo, hi) of level d* (the prefix
//           bucket of q[1..d*], Sec. 6.2) comes from the depth-1 buckets or
//           the 32-ary min tree over H.
//   fill    one warp per query: the first k - |A| ids of the level-d*
//           interval outside A, in ascending id order (an id-order probe, a
//           heavy trie node's precomputed list, or two sparse-table lists
//           and two partial blocks), then padding, into slots [|A|, k).
// Batches of up to 4,096 queries run the same stages per query in one fused
// kernel (a warp per query), as does the persistent work-queue worker.
#include <cuda/atomic>

#include <map>
#include <mutex>
#include <tuple>

#include "search.cuh"

namespace lcpk {

// ---- expansion chunk loads ----

// Loads the adjacent LCPs of up to 32 items on one side starting `n` items
// away from p (left: positions p-1-n-lane; right: positions p+n+lane).  Only
// LCPs: the ids of the few items that reach A are loaded when A is written.
template <bool LEFT>
__device__ __forceinline__ void issue_chunk(const DevIndex& ix, int p, int n, int avail, int l0,
                                            int& h, bool& ok) {
    const int lane = (int)lane_id();
    ok = n + lane < avail;
    h = 255;
    if (ok) {
        const int x = LEFT ? p - 1 - n - lane : p + n + lane;
        h = (n == 0 && lane == 0) ? l0 : (int)ix.H[LEFT ? x + 1 : x];
    }
}

// The items' LCPs with q (running minimum of H outward from p) into lam;
// returns the count.
__device__ __forceinline__ int finish_chunk(int& h, bool ok, int n, int avail, uint8_t* lam) {
    const unsigned lane = lane_id();
    if (n > 0) h = min(h, (int)lam[n - 1]);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, h, o);
        if (lane >= (unsigned)o) h = min(h, y);
    }
    if (ok) lam[n + lane] = (uint8_t)h;
    __syncwarp();
    return avail - n < 32 ? avail - n : 32;
}

// First round of a side: lane l holds the steps of items 2l and 2l + 1
// (255 where absent); they become the items' LCPs with q (the running
// minimum outward) and are stored into lam[2l], lam[2l + 1].
__device__ __forceinline__ void first_pair_scan(int& a, int& b, uint8_t* lam) {
    const unsigned lane = lane_id();
    int m = min(a, b);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, m, o);
        if (lane >= (unsigned)o) m = min(m, y);
    }
    int e = __shfl_up_sync(0xffffffffu, m, 1);  // the items before 2l
    if (lane == 0) e = 255;
    a = min(e, a);
    b = m;
    reinterpret_cast<uint16_t*>(lam)[lane] = (uint16_t)((a & 255) | ((b & 255) << 8));
}

// Id-order probe for a large tie level: walks ids 0, 1, 2, ... through pos[]
// (the low ids' positions are hot in L2 for every query), keeping ids whose
// sorted position lies in [lov, hiv) but outside A = [loc, hic).  Ascending
// by construction, written straight into the fill's output slots (oid and
// olcp point at the first).  At most 8 rounds of 256 ids; returns false when
// that did not find kp of them (the caller then uses the sparse-table path,
// which rewrites the same slots).
__device__ bool probe_ids(const DevIndex& ix, int64_t lov, int64_t hiv, int64_t loc, int64_t hic,
                          int kp, int32_t* __restrict__ oid, uint8_t* __restrict__ olcp, int dstar, int* ntake) {
    const unsigned lane = lane_id();
    const unsigned lt = lanemask_lt();
    int cnt = 0;
    int64_t base = 0;
    for (int round = 0; round < 8 && base < ix.N; ++round, base += 256) {
        int32_t ps[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int64_t id = base + lane + 32 * e;
            ps[e] = id < ix.N ? ix.pos[id] : -1;
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int64_t x = ps[e];
            const bool keep = x >= lov && x < hiv && (x < loc || x >= hic);
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            const int r = cnt + __popc(m & lt);
            if (keep && r < kp) {
                __stcs(oid + r, (int)(base + lane + 32 * e));
                __stcs(reinterpret_cast<char*>(olcp) + r, (char)dstar);
            }
            cnt += __popc(m);
        }
        if (cnt >= kp) {
            __syncwarp();
            *ntake = kp;
            return true;
        }
    }
    __syncwarp();
    if (base >= ix.N) {  // every id probed
        *ntake = cnt;
        return true;
    }
    return false;
}

// ---- the query's position: one lane per query ----

// Compares a sorted row with the query from word w0 on: -1 row < q, 0 equal,
// +1 row > q; *lcp = LCP(q, row) (given that words before w0 are equal).
__device__ __forceinline__ int lane_cmp_from(const DevIndex& ix, const uint64_t* __restrict__ row,
                                             const uint8_t* qrow, const RowFmt& qf, int w0, int* lcp) {
    for (int w = w0; w < ix.W; ++w) {
        const uint64_t a = row[w], b = pack_word(qrow, w, qf);
        if (a != b) {
            const int l = w * ix.tpw + (__clzll((long long)(a ^ b)) / ix.bits);
            *lcp = l < ix.L ? l : ix.L;
            return a < b ? -1 : 1;
        }
    }
    *lcp = ix.L;
    return 0;
}

// Algorithm 3's descent in array form, by one lane: the insertion point p
// (first row >= q) and the LCPs of q with rows p-1 and p (-1 where absent).
// The search starts inside the depth-1 bucket of q's first token (the rows
// before it are smaller than q, the rows after it larger).  Word 0 alone
// decides everything unless some row shares it with q; then a binary search
// inside that equal-head range compares the later words.
// [lo, hi]: a range known to hold the first position whose head is >= q0.
__device__ __forceinline__ void lane_locate_range(const DevIndex& ix, const uint8_t* qrow, const RowFmt& qf,
                                                  uint64_t q0, int lo, int hi, int64_t* p_out, int* lL_out,
                                                  int* lR_out) {
    const int N = (int)ix.N;  // positions are 32-bit: an index holds fewer than 2^30 rows
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ix.head[mid] < q0) lo = mid + 1;
        else hi = mid;
    }
    const int p0 = lo;
    int p1 = p0;
    if (p0 < N && ix.head[p0] == q0) {  // gallop to the end of the equal-head range
        int step = 1, last = p0;
        while (last + step < N && ix.head[last + step] == q0) {
            last += step;
            step <<= 1;
        }
        lo = last + 1;
        hi = last + step < N ? last + step : N;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (ix.head[mid] <= q0) lo = mid + 1;
            else hi = mid;
        }
        p1 = lo;
    }
    int p = p0;
    if (p1 > p0) {
        lo = p0;
        hi = p1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            int l;
            if (lane_cmp_from(ix, ix.rows + (size_t)mid * ix.W, qrow, qf, 1, &l) < 0) lo = mid + 1;
            else hi = mid;
        }
        p = lo;
    }
    int lL = -1, lR = -1;
    if (p > 0) {
        if (p - 1 >= p0) lane_cmp_from(ix, ix.rows + (size_t)(p - 1) * ix.W, qrow, qf, 1, &lL);
        else lL = __clzll((long long)(ix.head[p - 1] ^ q0)) / ix.bits;
    }
    if (p < N) {
        if (p < p1) lane_cmp_from(ix, ix.rows + (size_t)p * ix.W, qrow, qf, 1, &lR);
        else lR = __clzll((long long)(ix.head[p] ^ q0)) / ix.bits;
    }
    *p_out = p;
    *lL_out = lL;
    *lR_out = lR;
}

__device__ __forceinline__ void lane_locate(const DevIndex& ix, const uint8_t* qrow, const RowFmt& qf,
                                            uint64_t q0, int64_t* p_out, int* lL_out, int* lR_out) {
    const uint32_t t0 = (uint32_t)(q0 >> (64 - ix.bits));
    lane_locate_range(ix, qrow, qf, q0, ix.bkt[t0], ix.bkt[t0 + 1], p_out, lL_out, lR_out);
}

// Word 0 of a query; the load asks L2 for 64 bytes, not the row.
__device__ __forceinline__ uint64_t query_word0(const uint8_t* qrow, const RowFmt& qf) {
    if (qf.aligned8) {
        uint64_t q0;
        asm("ld.global.nc.L2::64B.u64 %0, [%1];" : "=l"(q0) : "l"(qrow));
        return msb_first(q0, qf.tb);
    }
    return pack_word(qrow, 0, qf);
}

// Lane per query with the top levels of the sorted array staged in shared
// memory: the CTA bulk-copies the sampled heads top[j] = head[j * N / T]
// (the TMA unit, one thread waiting with a bound), each lane binary-searches
// there the samples inside q's first-token bucket -- heads below q0 at j < c,
// so the first head >= q0 lies in (pos(c - 1), pos(c)] -- and finishes in L2
// over at most about N / T rows of the bucket instead of all of it.
constexpr int kStagedLocateThreads = 1024;

__global__ void __launch_bounds__(kStagedLocateThreads) k_topk_locate_staged(DevIndex ix,
                                                                            const uint8_t* __restrict__ queries,
                                                                            RowFmt qf, int64_t Q,
                                                                            QLoc* __restrict__ loc) {
    extern __shared__ __align__(128) uint64_t top_s[];
    __shared__ __align__(8) uint64_t tbar;
    const int T = ix.top_n;
    if (threadIdx.x == 0) {
        mbar_init(&tbar, 1);
        fence_proxy_async_smem();
        const uint32_t bytes = (uint32_t)((T * 8 + 15) & ~15);  // the table is padded to 16 bytes
        mbar_arrive_expect_tx(&tbar, bytes);
        bulk_g2s(top_s, ix.top, bytes, &tbar);
    }
    const bool ok = threadIdx.x != 0 || mbar_wait(&tbar, 0, kSpinLimit);
    if (__syncthreads_or(!ok)) {  // the copy never completed: report, let it land (bounded), leave
        if (threadIdx.x == 0) {
            flag_status(ix.status, DEV_TIMEOUT);
            mbar_wait(&tbar, 0, kSpinLimit);
        }
        __syncthreads();
        return;
    }
    const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= Q) return;
    const uint8_t* qrow = row_of(queries, qi, qf);
    const uint64_t q0 = query_word0(qrow, qf);
    const uint32_t t0 = (uint32_t)(q0 >> (64 - ix.bits));
    const int b0 = ix.bkt[t0], b1 = ix.bkt[t0 + 1];
    const int N = (int)ix.N;
    // c = number of sampled heads < q0: every sample before the bucket
    // (positions < b0: first token smaller) and none from its end on
    int c0 = (int)(((int64_t)b0 * T + N - 1) / N), c1 = (int)(((int64_t)b1 * T + N - 1) / N);
    if (c1 > T) c1 = T;
    while (c0 < c1) {
        const int m = (c0 + c1) >> 1;
        if (top_s[m] < q0) c0 = m + 1;
        else c1 = m;
    }
    const int lo = c0 == 0 ? 0 : (int)((int64_t)(c0 - 1) * N / T) + 1;
    const int hi = c0 == T ? N : (int)((int64_t)c0 * N / T);
    int64_t p;
    int lL, lR;
    lane_locate_range(ix, qrow, qf, q0, max(lo, b0), min(hi, b1), &p, &lL, &lR);
    QLoc r;
    r.p = p;
    r.lL = (int16_t)lL;
    r.lR = (int16_t)lR;
    r.tok0 = (int32_t)t0;
    loc[qi] = r;
}

__global__ void __launch_bounds__(256) k_topk_locate(DevIndex ix, const uint8_t* __restrict__ queries,
                                                     RowFmt qf, int64_t Q, QLoc* __restrict__ loc) {
    const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= Q) return;
    const uint8_t* qrow = row_of(queries, qi, qf);
    // word 0 alone decides most queries
    const uint64_t q0 = query_word0(qrow, qf);
    int64_t p;
    int lL, lR;
    lane_locate(ix, qrow, qf, q0, &p, &lL, &lR);
    QLoc r;
    r.p = p;
    r.lL = (int16_t)lL;
    r.lR = (int16_t)lR;
    r.tok0 = (int32_t)(q0 >> (64 - ix.bits));
    loc[qi] = r;
}

// Small batches: one warp per query.  The insertion point p (number of rows
// < q) is found by a 33-way search -- 32 probes per round, about log_33 N
// dependent loads instead of log_2 N -- so a batch of a few thousand queries
// spreads over every SM instead of a few CTAs.
__device__ __forceinline__ bool row_lt_query(const DevIndex& ix, int64_t m, const uint8_t* qrow,
                                             const RowFmt& qf, uint64_t q0) {
    const uint64_t h = ix.head[m];
    if (h != q0) return h < q0;
    int l;
    return lane_cmp_from(ix, ix.rows + m * ix.W, qrow, qf, 1, &l) < 0;
}

__device__ __forceinline__ int lcp_with_row(const DevIndex& ix, int64_t m, const uint8_t* qrow,
                                            const RowFmt& qf, uint64_t q0) {
    const uint64_t h = ix.head[m];
    if (h != q0) return __clzll((long long)(h ^ q0)) / ix.bits;
    int l;
    lane_cmp_from(ix, ix.rows + m * ix.W, qrow, qf, 1, &l);
    return l;
}

// One warp locates one query: p, lL, lR and the first token.
__device__ __forceinline__ QLoc warp_locate(const DevIndex& ix, const uint8_t* qrow, const RowFmt& qf) {
    const unsigned lane = lane_id();
    const uint64_t q0 = pack_word(qrow, 0, qf);
    const uint32_t t0 = (uint32_t)(q0 >> (64 - ix.bits));
    // rows < q form the prefix [0, p), p in [lo, hi]: within q's first-token bucket
    int64_t lo = ix.bkt[t0], hi = ix.bkt[t0 + 1];
    while (hi - lo > 32) {
        const int64_t m = lo + ((hi - lo) * (int64_t)(lane + 1)) / 33;
        const int c = __popc(__ballot_sync(0xffffffffu, row_lt_query(ix, m, qrow, qf, q0)));
        const int64_t mlast = __shfl_sync(0xffffffffu, m, c > 0 ? c - 1 : 0);
        const int64_t mnext = __shfl_sync(0xffffffffu, m, c < 32 ? c : 31);
        if (c > 0) lo = mlast + 1;
        if (c < 32) hi = mnext;
    }
    const bool t = lo + (int64_t)lane < hi && row_lt_query(ix, lo + lane, qrow, qf, q0);
    const int64_t p = lo + __popc(__ballot_sync(0xffffffffu, t));
    // neighbour LCPs: lane 0 takes row p - 1, lane 1 row p
    int l = -1;
    if (lane == 0 && p > 0) l = lcp_with_row(ix, p - 1, qrow, qf, q0);
    if (lane == 1 && p < ix.N) l = lcp_with_row(ix, p, qrow, qf, q0);
    QLoc r;
    r.p = p;
    r.lL = (int16_t)__shfl_sync(0xffffffffu, l, 0);
    r.lR = (int16_t)__shfl_sync(0xffffffffu, l, 1);
    r.tok0 = (int32_t)(q0 >> (64 - ix.bits));
    return r;
}

__global__ void __launch_bounds__(256) k_topk_locate_warp(DevIndex ix, const uint8_t* __restrict__ queries,
                                                          RowFmt qf, int64_t Q, QLoc* __restrict__ loc) {
    const int64_t qi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (qi >= Q) return;
    const QLoc r = warp_locate(ix, row_of(queries, qi, qf), qf);
    if (lane_id() == 0) loc[qi] = r;
}

// Batches up to this size locate with a warp per query (see above).
constexpr int64_t kWarpLocateMaxQ = 8192;

// ---- one query, whole warp ----

// What the second half of a query needs from the first: the level-d*
// interval, A's extent around p, and how many tie ids to add.
struct alignas(16) FillRec {
    int32_t lov, hiv;  // level-d* interval [lov, hiv)
    int32_t loc, hic;  // A = the items at positions [loc, hic) other than the tie level's
    int16_t nA, kp;    // |A|, tie ids to add
    int16_t dstar;
    int16_t pad;
    int32_t li;        // tie list of the level-d* node (-2: not looked up)
    int32_t pad2;
};

// First half of a query (expansion, d*, the level-d* interval, A ordered and
// written to output slots [0, |A|)).
template <typename KT, typename WA>
__device__ __forceinline__ FillRec topk_expand(const DevIndex& ix, WA& S, int p, int lL, int lR, int tok0,
                                               int k, int32_t* __restrict__ oid, uint8_t* __restrict__ olcp) {
    const unsigned lane = lane_id();
    const int N = (int)ix.N;  // positions are 32-bit: an index holds fewer than 2^30 rows
    // 3. expansion
    const int availL = p, availR = N - p;
    int nL = 0, nR = 0, dstar = 0;
    // the depth-1 bucket of q's first token, fetched early: d* is 1 for
    // about half of the queries, and these loads then cost no extra wait
    const int32_t bk0 = ix.bkt[tok0], bk1 = ix.bkt[tok0 + 1], bkl = ix.bkt_list[tok0];
    // and its depth-2 table (d* = 2 for about a fifth of the queries), with
    // the neighbour rows' first words that give q's second token
    const int32_t sti = ix.sub_idx ? ix.sub_idx[tok0] : -1;
    const uint64_t hnL = p > 0 ? ix.head[p - 1] : 0ull, hnR = p < N ? ix.head[p] : 0ull;
    // first round: 64 rows per side, every load in flight at once, lane l
    // holding items 2l and 2l + 1 of each side (one running-minimum scan a
    // side); the LCPs stay in registers too (-1 where absent) for the
    // decision below.  Left item i is row p-1-i, its step H[p-i]; right item
    // i is row p+i, its step H[p+i]; item 0's step is the neighbour's LCP.
    int vL0, vL1, vR0, vR1;
    {
        const int i0 = 2 * (int)lane, i1 = i0 + 1;
        const bool okL0 = i0 < availL, okL1 = i1 < availL, okR0 = i0 < availR, okR1 = i1 < availR;
        int hL0 = okL0 ? (i0 == 0 ? lL : (int)ix.H[p - i0]) : 255;
        int hL1 = okL1 ? (int)ix.H[p - i1] : 255;
        int hR0 = okR0 ? (i0 == 0 ? lR : (int)ix.H[p + i0]) : 255;
        int hR1 = okR1 ? (int)ix.H[p + i1] : 255;
        first_pair_scan(hL0, hL1, S.llam);
        first_pair_scan(hR0, hR1, S.rlam);
        __syncwarp();
        nL = availL < 64 ? availL : 64;
        nR = availR < 64 ? availR : 64;
        vL0 = okL0 ? hL0 : -1;
        vL1 = okL1 ? hL1 : -1;
        vR0 = okR0 ? hR0 : -1;
        vR1 = okR1 ? hR1 : -1;
    }
    // Decision after the first round, in registers: the LCP bound of the
    // unloaded items on each side is the last loaded LCP there; if at least
    // k loaded items reach the larger bound F (or nothing is left), d* is
    // the k-th largest loaded LCP -- found by bisection on the value with
    // ballot counts -- and A's and the tie level's counts follow by ballots.
    // Otherwise (about one query in seven) the expansion continues below.
    bool decided = false;
    int aL = 0, aR = 0, vL = 0, vR = 0;
    {
        auto at = [&](int v0, int v1, int i) {  // item i of a side (i < 64): lane i / 2
            const int a = __shfl_sync(0xffffffffu, v0, i >> 1);
            const int b = __shfl_sync(0xffffffffu, v1, i >> 1);
            return (i & 1) ? b : a;
        };
        auto cnt_ge = [&](int v) {  // absent items hold -1
            const unsigned c = (unsigned)(vL0 >= v) + (unsigned)(vL1 >= v) + (unsigned)(vR0 >= v) + (unsigned)(vR1 >= v);
            return (int)__reduce_add_sync(0xffffffffu, c);
        };
        const int bL = nL < availL ? at(vL0, vL1, nL - 1) : -1;
        const int bR = nR < availR ? at(vR0, vR1, nR - 1) : -1;
        const int F = bL > bR ? bL : bR;
        bool ok = F < 0;
        if (!ok) ok = cnt_ge(F) >= k;  // loaded items with LCP >= F (every loaded item of F's side qualifies)
        if (ok) {
            if (nL + nR >= k) {
                // largest v with cnt_ge(v) >= k: at least F (when F >= 0,
                // cnt_ge(F) >= k was just checked) and at most the largest
                // loaded LCP, max(lL, lR)
                int lo = F > 0 ? F : 0, hi = (lL > lR ? lL : lR) + 1;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (cnt_ge(mid) >= k) lo = mid;
                    else hi = mid;
                }
                dstar = lo;
            } else {
                dstar = 0;
            }
            aL = (int)__reduce_add_sync(0xffffffffu, (unsigned)(vL0 > dstar) + (unsigned)(vL1 > dstar));
            aR = (int)__reduce_add_sync(0xffffffffu, (unsigned)(vR0 > dstar) + (unsigned)(vR1 > dstar));
            vL = (int)__reduce_add_sync(0xffffffffu, (unsigned)(vL0 >= dstar) + (unsigned)(vL1 >= dstar));
            vR = (int)__reduce_add_sync(0xffffffffu, (unsigned)(vR0 >= dstar) + (unsigned)(vR1 >= dstar));
            decided = true;
        }
    }
    for (; !decided;) {
        const int bL = nL < availL ? (int)S.llam[nL - 1] : -1;
        const int bR = nR < availR ? (int)S.rlam[nR - 1] : -1;
        const int F = bL > bR ? bL : bR;
        if (F < 0) {  // every item loaded
            dstar = nL + nR >= k ? kth_largest(S.llam, nL, S.rlam, nR, k) : 0;
            break;
        }
        // loaded items with LCP >= F (the side holding F counts entirely)
        const int cnt = bL >= bR ? nL + count_ge(S.rlam, nR, F) : nR + count_ge(S.llam, nL, F);
        if (cnt >= k) {
            dstar = kth_largest(S.llam, nL, S.rlam, nR, k);
            break;
        }
        int h;
        bool ok;
        if (bL >= bR) {
            if (nL + 32 > kSide) {
                flag_status(ix.status, DEV_BAD);
                break;
            }
            issue_chunk<true>(ix, p, nL, availL, lL, h, ok);
            nL += finish_chunk(h, ok, nL, availL, S.llam);
        } else {
            if (nR + 32 > kSide) {
                flag_status(ix.status, DEV_BAD);
                break;
            }
            issue_chunk<false>(ix, p, nR, availR, lR, h, ok);
            nR += finish_chunk(h, ok, nR, availR, S.rlam);
        }
    }
    // A = loaded items with LCP > d*; interval [lov, hiv) of level d*.
    // (Past the first round) counts of loaded items with LCP > d* (aX) and
    // >= d* (vX) per side, by ballots over the non-increasing LCP arrays.
    if (!decided) {
        for (int b = 0; b < nL; b += 32) {
            const int t = b + (int)lane;
            const int l = t < nL ? (int)S.llam[t] : -1;
            aL += __popc(__ballot_sync(0xffffffffu, l > dstar));
            vL += __popc(__ballot_sync(0xffffffffu, l >= dstar));
        }
        for (int b = 0; b < nR; b += 32) {
            const int t = b + (int)lane;
            const int l = t < nR ? (int)S.rlam[t] : -1;
            aR += __popc(__ballot_sync(0xffffffffu, l > dstar));
            vR += __popc(__ballot_sync(0xffffffffu, l >= dstar));
        }
    }
    const int nA = aL + aR;
    int lov = 0, hiv = N;
    int li = -2;  // tie list of the level-d* node (-2: not looked up yet)
    if (dstar == 1) {  // depth-1 bucket of q's first token (fetched above)
        lov = bk0;
        hiv = bk1;
        li = bkl;
    } else if (dstar > 1) {
        const bool knownL = vL < nL || nL == availL;
        const bool knownR = vR < nR || nR == availR;
        if (dstar == 2 && sti >= 0 && !(knownL && knownR)) {
            // the depth-2 bucket of q's first two tokens (those of the
            // neighbour row with the larger LCP, which is >= 2)
            const uint32_t t1 =
                (uint32_t)((lL >= lR ? hnL : hnR) >> (64 - 2 * ix.bits)) & ((1u << ix.bits) - 1);
            const int2 run = ix.sub[((int64_t)sti << ix.bits) + t1];
            lov = knownL ? p - vL : run.x;
            hiv = knownR ? p + vR : run.y;
        } else if (dstar <= ix.tpw && !(knownL && knownR)) {
            // the run lies in word 0: searches over head inside the bucket;
            // a neighbour of p with LCP >= d* gives the run's masked word 0
            const uint64_t mask = ~0ull << (64 - dstar * ix.bits);
            const uint64_t key = ix.head[lL >= lR ? p - 1 : p] & mask;
            int xl = 0, xr = N;
            head_bounds(ix, bk0, bk1, p - nL, p + nR, key, mask, !knownL, !knownR, &xl, &xr);
            lov = knownL ? p - vL : xl;
            hiv = knownR ? p + vR : xr;
        } else {
            int xl = -1, xr = N;
            find_bounds(ix, p - nL, !knownL, p + nR, !knownR, dstar, &xl, &xr);
            lov = knownL ? p - vL : (xl < 0 ? 0 : xl);
            hiv = knownR ? p + vR : xr;
        }
    }
    const int nT = (hiv - lov) - nA;
    int kp = k - nA;
    if (kp > nT) kp = nT;
    // 5a. A sorted by (LCP desc, id asc) into slots [0, nA)
    if (nA > 0) {
        if (nA <= 32) rank_and_write_A<KT>(S, ix.ids, p, aL, nA, oid, olcp);
        else if (nA <= 64) sort_and_write_A<2, KT>(S, ix.ids, p, aL, nA, oid, olcp);
        else sort_and_write_A<4, KT>(S, ix.ids, p, aL, nA, oid, olcp);
    }
    FillRec r;
    r.lov = lov;
    r.hiv = hiv;
    r.loc = p - aL;
    r.hic = p + aR;
    r.nA = (int16_t)nA;
    r.kp = (int16_t)(kp > 0 ? kp : 0);
    r.dstar = (int16_t)dstar;
    r.li = li;
    r.pad = 0;
    r.pad2 = 0;
    return r;
}

// Second half of a query: 4. the tie fill (first kp ids of the level-d*
// interval outside A) and 5b. slots [nA, k): the fill, then padding.
// Writes the kept ids of v (ascending across e, then lanes) into slots
// 0, 1, ... of the fill's output (at most kp of them); returns how many.
__device__ __forceinline__ int fill_write4(const uint32_t (&v)[4], const bool (&keep)[4], int kp,
                                           int32_t* __restrict__ oid, uint8_t* __restrict__ olcp, int dstar) {
    const unsigned ltm = lanemask_lt();
    int cnt = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const unsigned m = __ballot_sync(0xffffffffu, keep[e]);
        const int r = cnt + __popc(m & ltm);
        if (keep[e] && r < kp) {
            __stcs(oid + r, (int)v[e]);
            __stcs(reinterpret_cast<char*>(olcp) + r, (char)dstar);
        }
        cnt += __popc(m);
    }
    return cnt < kp ? cnt : kp;
}

template <typename WA>
__device__ __forceinline__ void topk_fill(const DevIndex& ix, WA& S, const FillRec& r, int k,
                                          int32_t* __restrict__ oid, uint8_t* __restrict__ olcp) {
    const unsigned lane = lane_id();
    const int64_t N = ix.N;
    const int64_t lov = r.lov, hiv = r.hiv, loc = r.loc, hic = r.hic;
    const int nA = r.nA, kp = r.kp, dstar = r.dstar;
    const int64_t nT = (hiv - lov) - nA;
    int li = r.li;
    int ntake = 0;
    bool filled = kp <= 0;
    // a tie level holding a large share of all rows: probe ids in order
    // (expected <= 6 chunks of 128 ids)
    if (!filled && (int64_t)kp * N <= nT * 768)
        filled = probe_ids(ix, lov, hiv, loc, hic, kp, oid + nA, olcp + nA, dstar, &ntake);
    // a heavy trie node: its precomputed K smallest ids (with their sorted
    // positions), minus A's members
    if (!filled && hiv - lov > kBlk) {
        if (li == -2) li = ix.tbl ? ix.tbl[((lov + kBlk - 1) / kBlk) * ix.L1 + dstar] : -1;
        if (li >= 0) {
            const uint32_t* list = ix.tlists + (size_t)li * ix.K;
            const int32_t* lpos = ix.tlpos + (size_t)li * ix.K;
            const int need = nA + kp;
            uint32_t v[4];
            int32_t ps[4];
            bool keep[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int t = (int)lane + 32 * e;
                v[e] = t < need ? list[t] : kInf;
                ps[e] = t < need ? lpos[t] : -1;
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) keep[e] = v[e] != kInf && (ps[e] < loc || ps[e] >= hic);
            // the kept ids (ascending) straight into slots nA, nA + 1, ...
            ntake = fill_write4(v, keep, kp, oid + nA, olcp + nA, dstar);
            filled = true;
        }
    }
    if (!filled) {
        const int need = nA + kp;
        const int cm = smallest_ids(ix, lov, hiv, need, S);
        uint32_t v[4];
        bool keep[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int t = (int)lane + 32 * e;
            v[e] = t < cm ? S.src[0][t] : kInf;
        }
        int64_t ps[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) ps[e] = v[e] != kInf ? (int64_t)ix.pos[v[e]] : -1;
#pragma unroll
        for (int e = 0; e < 4; ++e) keep[e] = v[e] != kInf && (ps[e] < loc || ps[e] >= hic);
        __syncwarp();
        ntake = fill_write4(v, keep, kp, oid + nA, olcp + nA, dstar);
    }
    // slots past the fill: padding
    for (int t = nA + ntake + (int)lane; t < k; t += 32) {
        __stcs(oid + t, -1);
        __stcs(reinterpret_cast<char*>(olcp) + t, (char)0);
    }
    __syncwarp();
}

// One query, whole warp (the persistent worker runs both halves in place).
template <typename KT>
__device__ __forceinline__ void topk_one(const DevIndex& ix, QWarp& S, int64_t p, int lL, int lR, int tok0, int k,
                                         int32_t* __restrict__ oid, uint8_t* __restrict__ olcp) {
    const FillRec r = topk_expand<KT>(ix, S, (int)p, lL, lR, tok0, k, oid, olcp);
    topk_fill(ix, S, r, k, oid, olcp);
}

// Batched search, second and third kernels: the two halves of every query,
// split so that each kernel's code stays small enough for the instruction
// cache (warps of one kernel sit in different phases at once).  The answer
// kernel runs 12 CTAs (48 warps) per multiprocessor: its warps wait on
// dependent L2 loads, and the extra warps cover them (0.706 -> 0.684 ms at
// 1M queries, measured; 16 CTAs spill and are slower).
template <typename KT>
__global__ void __launch_bounds__(kSearchWarps * 32, 12) k_topk_answer(DevIndex ix, const QLoc* __restrict__ loc,
                                                                      int64_t Q, int k, int qpw,
                                                                      int32_t* __restrict__ out_ids,
                                                                      uint8_t* __restrict__ out_lcp,
                                                                      FillRec* __restrict__ recs) {
    __shared__ AWarp sm[kSearchWarps];
    const int warp = threadIdx.x >> 5;
    AWarp& S = sm[warp];
    const int64_t wq0 = ((int64_t)blockIdx.x * kSearchWarps + warp) * qpw;
    for (int j = 0; j < qpw; ++j) {
        const int64_t qi = wq0 + j;
        if (qi >= Q) break;
        const QLoc r = loc[qi];
        const FillRec f = topk_expand<KT>(ix, S, (int)r.p, r.lL, r.lR, r.tok0, k, out_ids + qi * k, out_lcp + qi * k);
        if (lane_id() == 0) recs[qi] = f;
    }
}

__global__ void __launch_bounds__(kSearchWarps * 32, 10) k_topk_fill(DevIndex ix, const FillRec* __restrict__ recs,
                                                                    int64_t Q, int k, int qpw,
                                                                    int32_t* __restrict__ out_ids,
                                                                    uint8_t* __restrict__ out_lcp) {
    __shared__ FWarp sm[kSearchWarps];
    const int warp = threadIdx.x >> 5;
    FWarp& S = sm[warp];
    const int64_t wq0 = ((int64_t)blockIdx.x * kSearchWarps + warp) * qpw;
    for (int j = 0; j < qpw; ++j) {
        const int64_t qi = wq0 + j;
        if (qi >= Q) break;
        const FillRec f = recs[qi];
        topk_fill(ix, S, f, k, out_ids + qi * k, out_lcp + qi * k);
    }
}

// Small batches: one kernel, a warp per query -- locate (33-way search),
// expansion and tie fill in place -- so a batch costs one launch and no
// scratch instead of three launches and the per-query records.
template <typename KT>
__global__ void __launch_bounds__(kSearchWarps * 32) k_topk_fused(DevIndex ix, const uint8_t* __restrict__ queries,
                                                                  RowFmt qf, int64_t Q, int k,
                                                                  int32_t* __restrict__ out_ids,
                                                                  uint8_t* __restrict__ out_lcp) {
    __shared__ QWarp sm[kSearchWarps];
    const int warp = threadIdx.x >> 5;
    const int64_t qi = (int64_t)blockIdx.x * kSearchWarps + warp;
    if (qi >= Q) return;
    const QLoc r = warp_locate(ix, row_of(queries, qi, qf), qf);
    topk_one<KT>(ix, sm[warp], r.p, r.lL, r.lR, r.tok0, k, out_ids + qi * k, out_lcp + qi * k);
}

// ---- persistent worker ----

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Lane 0: claims the next task id, or returns -1 after idle_ns without one
// (or at once when stop is set).  Claims are fetch-and-adds on a device
// counter, taken only when a task looks available; a warp that loses that
// race holds an id past the published count and waits for it to be
// published.  If it gives up first, the id is recorded in min_abandoned, and
// the last warp to leave the launch rewinds the counter to it, so the next
// launch claims it again; ids processed meanwhile are skipped there (see
// take_task).  Every wait is bounded: by the idle clock, and by kSpinLimit
// iterations.
__device__ int64_t claim_task(const QueueArgs& a) {
    const volatile int64_t* pub = &a.ctl->published;
    const volatile int32_t* stop = &a.ctl->stop;
    long long t0 = global_ns();
    unsigned ns = 32;
    long long spin = 0;
    for (; spin < kSpinLimit; ++spin) {  // until a task looks available
        if (*(volatile int64_t*)a.claimed < *pub) break;
        if (*stop || global_ns() - t0 > a.idle_ns) return -1;
        __nanosleep(ns);
        if (ns < 8192) ns <<= 1;
    }
    if (spin >= kSpinLimit) {
        flag_status(a.status, DEV_TIMEOUT);
        return -1;
    }
    const int64_t t = (int64_t)atomicAdd((unsigned long long*)a.claimed, 1ull);
    t0 = global_ns();
    ns = 32;
    for (; spin < kSpinLimit; ++spin) {  // until it is published
        if (t < *pub) {
            __threadfence();  // records are read after the count that covers them
            return t;
        }
        if (*stop || global_ns() - t0 > a.idle_ns) break;
        __nanosleep(ns);
        if (ns < 8192) ns <<= 1;
    }
    atomicMin((long long*)a.min_abandoned, (long long)t);
    if (spin >= kSpinLimit) flag_status(a.status, DEV_TIMEOUT);
    return -1;
}

// A task id is answered once: the ring slot remembers the largest id taken
// from it (ids of one slot only grow: t, t + tcap, ...).
__device__ __forceinline__ bool take_task(const QueueArgs& a, int64_t t) {
    return (int64_t)atomicMax((long long*)&a.taken[t % a.tcap], (long long)t) < t;
}

// The last warp of a launch to leave: rewind past abandoned ids.
__device__ void leave_launch(const QueueArgs& a) {
    const unsigned total = gridDim.x * kSearchWarps;
    if (atomicAdd(a.exited, 1u) != total - 1) return;
    const int64_t m = *(volatile int64_t*)a.min_abandoned;
    if (m < *(volatile int64_t*)a.claimed) *(volatile int64_t*)a.claimed = m;
    *(volatile int64_t*)a.min_abandoned = INT64_MAX;
    *(volatile unsigned*)a.exited = 0;
    __threadfence();
}

// Warps claim tasks until the queue stays empty for idle_ns.  A task's
// request is copied into the warp's shared memory (index snapshot and
// pointers), then each query is located and answered exactly as by
// lcp_topk_batch.  The warp that finishes a request's last task resets its
// counter and publishes the ticket to host memory after a system fence.
__global__ void __launch_bounds__(kSearchWarps * 32, 8) k_queue_worker(QueueArgs a) {
    __shared__ QWarp sm[kSearchWarps];
    __shared__ QReq rq[kSearchWarps];
    const int warp = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    QWarp& S = sm[warp];
    QReq& R = rq[warp];
    for (;;) {
        int64_t t = 0;
        bool mine = false;
        if (lane == 0) {
            t = claim_task(a);
            if (t < 0) leave_launch(a);
            else mine = take_task(a, t);
        }
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t < 0) break;
        if (!__shfl_sync(0xffffffffu, mine, 0)) continue;  // answered before a rewind
        QTask task;
        {
            const volatile QTask* tw = &a.tasks[t % a.tcap];
            task.q0 = tw->q0;
            task.q1 = tw->q1;
            task.slot = tw->slot;
        }
        {  // the request record, copied word by word by the warp
            const volatile uint64_t* src = reinterpret_cast<const volatile uint64_t*>(&a.reqs[task.slot]);
            uint64_t* dst = reinterpret_cast<uint64_t*>(&R);
            for (int w = (int)lane; w < (int)(sizeof(QReq) / 8); w += 32) dst[w] = src[w];
        }
        __syncwarp();
        const bool wide = R.ix.N > (1ll << 24);
        for (int64_t qi = task.q0; qi < task.q1; ++qi) {
            const QLoc r = warp_locate(R.ix, row_of(R.queries, qi, R.qf), R.qf);
            int32_t* oid = R.out_ids + qi * R.k;
            uint8_t* olcp = R.out_lcp + qi * R.k;
            if (wide) topk_one<uint64_t>(R.ix, S, r.p, r.lL, r.lR, r.tok0, R.k, oid, olcp);
            else topk_one<uint32_t>(R.ix, S, r.p, r.lL, r.lR, r.tok0, R.k, oid, olcp);
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) {
            const int n = atomicAdd(&a.done_count[task.slot], 1);
            if (n == R.ntasks - 1) {
                a.done_count[task.slot] = 0;
                __threadfence_system();
                cuda::atomic_ref<uint64_t, cuda::thread_scope_system>(a.done[task.slot])
                    .store(R.ticket, cuda::memory_order_release);
            }
        }
        __syncwarp();
    }
}

}  // namespace lcpk

namespace lcph {
using namespace lcpk;

// ---- launch shapes: heuristics, overridden by autotuned entries ----

namespace {
struct TuneKey {
    int nlog, L, tb, qlog, kb;
    bool operator<(const TuneKey& o) const {
        return std::tie(nlog, L, tb, qlog, kb) < std::tie(o.nlog, o.L, o.tb, o.qlog, o.kb);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, SearchShape> g_tune;

int ilog2(int64_t v) { return v <= 1 ? 0 : 63 - __builtin_clzll((unsigned long long)v); }
TuneKey tune_key(const lcp_index_s* x, int64_t Q, int k) {
    return {ilog2(x->N), x->L, x->tb, ilog2(Q), k <= 1 ? 0 : (k <= 16 ? 1 : (k <= 64 ? 2 : 3))};
}
}  // namespace

// Batches up to this size are answered by the fused kernel by default.
constexpr int64_t kFusedMaxQ = 4096;

SearchShape default_shape(int64_t Q) {
    SearchShape sh;
    sh.fused = Q <= kFusedMaxQ ? 1 : 0;
    sh.locate_warp = Q <= kWarpLocateMaxQ ? 1 : 0;
    // queries per warp: at most 8 (measured best for large batches: enough
    // warps for an even tail); fewer for small batches so that the batch
    // still spreads over every SM
    const int64_t full = (int64_t)sm_count() * 32;  // resident warps at full occupancy
    int64_t qpw = (Q + full - 1) / full;
    sh.qpw = (int)(qpw < 1 ? 1 : (qpw > 8 ? 8 : qpw));
    return sh;
}

SearchShape search_shape(const lcp_index_s* x, int64_t Q, int k) {
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(tune_key(x, Q, k));
        if (it != g_tune.end()) return it->second;
    }
    return default_shape(Q);
}

void set_search_shape(const lcp_index_s* x, int64_t Q, int k, const SearchShape& sh) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[tune_key(x, Q, k)] = sh;
}

void launch_locate(const DevIndex& ix, const uint8_t* q, const RowFmt& qf, int64_t Q, QLoc* loc, cudaStream_t s,
                   int warp_mode) {
    if (warp_mode < 0) warp_mode = Q <= kWarpLocateMaxQ ? 1 : 0;
    if (warp_mode == 1) {
        LCP_TIMED_LAUNCH(k_topk_locate_warp, (unsigned)((Q + 7) / 8), 256, 0, s, ix, q, qf, Q, loc);
    } else if (warp_mode == 2 && ix.top_n > 0) {
        const size_t smem = (size_t)((ix.top_n * 8 + 15) & ~15);
        LCP_TIMED_LAUNCH(k_topk_locate_staged, (unsigned)((Q + kStagedLocateThreads - 1) / kStagedLocateThreads),
                         kStagedLocateThreads, smem, s, ix, q, qf, Q, loc);
    } else {
        LCP_TIMED_LAUNCH(k_topk_locate, (unsigned)((Q + 255) / 256), 256, 0, s, ix, q, qf, Q, loc);
    }
}

void launch_queue_worker(const QueueArgs& a, unsigned grid, cudaStream_t s) {
    LCP_LAUNCH(k_queue_worker, grid, kSearchWarps * 32, 0, s, a);
}

int topk_batch_device(lcp_index_s* x, const void* d_queries, int64_t Q, int k, int32_t* out_ids,
                      uint8_t* out_lcp, cudaStream_t s, void* loc_scratch, const SearchShape* shape) {
    if (Q <= 0) return LCP_OK;
    if (x->N == 0) {
        LCP_CUDA_TRY(cudaMemsetAsync(out_ids, 0xFF, sizeof(int32_t) * (size_t)Q * k, s));
        LCP_CUDA_TRY(cudaMemsetAsync(out_lcp, 0, (size_t)Q * k, s));
        return LCP_OK;
    }
    DevIndex ix = dev_view(x);
    RowFmt qf = make_fmt(x->tb, x->L, d_queries);
    const uint8_t* q = reinterpret_cast<const uint8_t*>(d_queries);
    const SearchShape sh = shape ? *shape : search_shape(x, Q, k);
    if (sh.fused) {
        const unsigned fgrid = (unsigned)((Q + kSearchWarps - 1) / kSearchWarps);
        if (x->N <= (1ll << 24))
            LCP_TIMED_LAUNCH(k_topk_fused<uint32_t>, fgrid, kSearchWarps * 32, 0, s, ix, q, qf, Q, k, out_ids, out_lcp);
        else
            LCP_TIMED_LAUNCH(k_topk_fused<uint64_t>, fgrid, kSearchWarps * 32, 0, s, ix, q, qf, Q, k, out_ids, out_lcp);
        return LCP_OK;
    }
    // position records: the caller's buffer (a captured graph must not
    // allocate), else stream-ordered scratch
    QLoc* loc = reinterpret_cast<QLoc*>(loc_scratch);
    const bool own = loc == nullptr;
    if (own) LCP_CUDA_TRY(cudaMallocAsync((void**)&loc, search_scratch_bytes(Q), s));
    launch_locate(ix, q, qf, Q, loc, s, sh.locate_warp);
    const int qpw = sh.qpw;
    const int64_t warps = (Q + qpw - 1) / qpw;
    const unsigned grid = (unsigned)((warps + kSearchWarps - 1) / kSearchWarps);
    FillRec* recs = reinterpret_cast<FillRec*>(loc + Q);  // after the position records (16-byte aligned)
    if (x->N <= (1ll << 24)) {
        LCP_TIMED_LAUNCH(k_topk_answer<uint32_t>, grid, kSearchWarps * 32, 0, s, ix, loc, Q, k, qpw, out_ids,
                         out_lcp, recs);
    } else {
        LCP_TIMED_LAUNCH(k_topk_answer<uint64_t>, grid, kSearchWarps * 32, 0, s, ix, loc, Q, k, qpw, out_ids,
                         out_lcp, recs);
    }
    LCP_TIMED_LAUNCH(k_topk_fill, grid, kSearchWarps * 32, 0, s, ix, recs, Q, k, qpw, out_ids, out_lcp);
    if (own) LCP_CUDA_TRY(cudaFreeAsync(loc, s));
    return LCP_OK;
}

size_t search_scratch_bytes(int64_t Q) { return (sizeof(QLoc) + sizeof(FillRec)) * (size_t)(Q > 0 ? Q : 1); }

}  // namespace lcph
