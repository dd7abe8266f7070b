// Indexed batched top-k (Algorithm 3 + CollectTopK / CollectTopKOptimized,
// returning the order of the Definition "Top-k LCP Retrieval").
//
// Per warp, 32 queries:
//   1. lane-per-query binary search on the L2-resident head array (word 0 of
//      every sorted row): p0 = first row with head >= q0, p1 = first with
//      head > q0.  32 independent searches per warp keep many probes in flight.
//   then warp-per-query, for each of the 32:
//   2. lower bound p inside [p0, p1) on the full rows (one coalesced row per
//      probe), and lL = LCP(q, row p-1), lR = LCP(q, row p).  max(lL, lR) is
//      the descent depth d of Algorithm 3.
//   3. expansion: along each side the LCP of row j with q is the running
//      minimum of H towards p (descent lemma, App. A).  32-item chunks are
//      loaded from the side whose next LCP is larger, until the k-th largest
//      loaded LCP d* is >= everything not yet loaded.  Items with LCP > d*
//      (fewer than k; the set A = interval of level d*+1) are all taken.
//   4. the interval [lo, hi) of level d* (the prefix bucket of q[1..d*],
//      Sec. 6.2) is closed with the 32-ary min tree over H, its smallest ids
//      come from two partial blocks and two sparse-table lists, A's members
//      are skipped, and the first k - |A| fill the remaining slots in
//      ascending id order (ties by index).
//   5. A is sorted by (LCP desc, id asc) in shared memory and the row of k
//      (id, lcp) results is written with coalesced stores.
#include "index.cuh"

namespace lcpk {

constexpr int kSearchWarps = 4;
constexpr int kMaxW = 64;
constexpr int kKMax = LCP_INDEX_MAX_K;
constexpr int kSide = kKMax + 64;  // loaded items per side never exceed k + 32

struct alignas(16) QWarp {
    uint64_t q[kMaxW];
    uint64_t akey[kKMax];
    uint32_t lid[kSide];
    uint32_t rid[kSide];
    uint32_t src[4][kKMax];
    uint32_t m1[2 * kKMax];
    uint32_t m2[2 * kKMax];
    uint8_t llam[kSide];
    uint8_t rlam[kSide];
};

// ---- warp-wide comparisons against the query held in shared memory ----

// -1 if row < q, 0 if equal, +1 if row > q; *lcp receives LCP(q, row).
__device__ __forceinline__ int warp_cmp_row(const uint64_t* __restrict__ row, const uint64_t* q,
                                            const DevIndex& ix, int* lcp) {
    const unsigned lane = lane_id();
    for (int w0 = 0; w0 < ix.W; w0 += 32) {
        int w = w0 + (int)lane;
        uint64_t a = 0, b = 0;
        if (w < ix.W) {
            a = row[w];
            b = q[w];
        }
        unsigned ne = __ballot_sync(0xffffffffu, a != b);
        if (ne) {
            int f = __ffs(ne) - 1;
            uint64_t ra = __shfl_sync(0xffffffffu, a, f);
            uint64_t qb = __shfl_sync(0xffffffffu, b, f);
            int l = (w0 + f) * ix.tpw + (__clzll((long long)(ra ^ qb)) / ix.bits);
            *lcp = l < ix.L ? l : ix.L;
            return ra < qb ? -1 : 1;
        }
    }
    *lcp = ix.L;
    return 0;
}

// ---- min tree over H: next / previous position with H < d ----

__device__ __forceinline__ const uint8_t* hlevel(const DevIndex& ix, int lev) {
    return lev == 0 ? ix.H : ix.hmin + ix.hoff[lev];
}

// Smallest x >= from with H[x] < d, or N.
__device__ int64_t next_less(const DevIndex& ix, int64_t from, int d) {
    const unsigned lane = lane_id();
    if (from >= ix.N) return ix.N;
    int64_t idx = from;
    int lev = 0;
    for (;;) {
        const uint8_t* arr = hlevel(ix, lev);
        int64_t len = ix.hlen[lev];
        int64_t g0 = (idx >> 5) << 5;
        int64_t e = g0 + lane;
        bool ok = e >= idx && e < len && (int)arr[e] < d;
        unsigned m = __ballot_sync(0xffffffffu, ok);
        if (m) {
            idx = g0 + __ffs(m) - 1;
            break;
        }
        if (lev == ix.hlev) return ix.N;
        idx = (idx >> 5) + 1;
        ++lev;
        if (idx >= ix.hlen[lev]) return ix.N;
    }
    while (lev > 0) {
        --lev;
        const uint8_t* arr = hlevel(ix, lev);
        int64_t len = ix.hlen[lev];
        int64_t g0 = idx << 5;
        int64_t e = g0 + lane;
        bool ok = e < len && (int)arr[e] < d;
        unsigned m = __ballot_sync(0xffffffffu, ok);
        if (!m) {  // cannot happen for a consistent tree
            flag_status(ix.status, DEV_BAD);
            return ix.N;
        }
        idx = g0 + __ffs(m) - 1;
    }
    return idx;
}

// Largest x <= from with H[x] < d, or -1.
__device__ int64_t prev_less(const DevIndex& ix, int64_t from, int d) {
    const unsigned lane = lane_id();
    if (from < 0) return -1;
    int64_t idx = from;
    int lev = 0;
    for (;;) {
        const uint8_t* arr = hlevel(ix, lev);
        int64_t len = ix.hlen[lev];
        int64_t g0 = (idx >> 5) << 5;
        int64_t e = g0 + lane;
        bool ok = e <= idx && e < len && (int)arr[e] < d;
        unsigned m = __ballot_sync(0xffffffffu, ok);
        if (m) {
            idx = g0 + 31 - __clz(m);
            break;
        }
        if (lev == ix.hlev) return -1;
        idx = (idx >> 5) - 1;
        ++lev;
        if (idx < 0) return -1;
    }
    while (lev > 0) {
        --lev;
        const uint8_t* arr = hlevel(ix, lev);
        int64_t len = ix.hlen[lev];
        int64_t g0 = idx << 5;
        int64_t e = g0 + lane;
        bool ok = e < len && (int)arr[e] < d;
        unsigned m = __ballot_sync(0xffffffffu, ok);
        if (!m) {
            flag_status(ix.status, DEV_BAD);
            return -1;
        }
        idx = g0 + 31 - __clz(m);
    }
    return idx;
}

// ---- small warp utilities over shared memory ----

// Number of leading entries of a non-increasing array that are >= d.
__device__ __forceinline__ int count_ge(const uint8_t* a, int n, int d) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((int)a[mid] >= d) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// k-th largest value of the union of two non-increasing arrays (1 <= k <= na+nb).
__device__ __forceinline__ int kth_largest(const uint8_t* a, int na, const uint8_t* b, int nb, int k) {
    int lo = k - nb > 0 ? k - nb : 0;
    int hi = k < na ? k : na;
    while (lo < hi) {
        int i = (lo + hi) >> 1;
        if (a[i] > b[k - i - 1]) lo = i + 1;
        else hi = i;
    }
    int i = lo, j = k - lo;
    int va = i > 0 ? (int)a[i - 1] : 1 << 20;
    int vb = j > 0 ? (int)b[j - 1] : 1 << 20;
    return va < vb ? va : vb;
}

// First nout entries of the merge of sorted a[0..na) and b[0..nb).
__device__ __forceinline__ void warp_merge(const uint32_t* a, int na, const uint32_t* b, int nb,
                                           uint32_t* out, int nout) {
    const int lane = (int)lane_id();
    int per = (nout + 31) >> 5;
    int d0 = lane * per;
    if (d0 < nout) {
        int lo = d0 - nb > 0 ? d0 - nb : 0, hi = d0 < na ? d0 : na;
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (a[mid] <= b[d0 - 1 - mid]) lo = mid + 1;
            else hi = mid;
        }
        int i = lo, j = d0 - lo;
        int end = d0 + per < nout ? d0 + per : nout;
        for (int t = d0; t < end; ++t) {
            bool takeA = (i < na) && (j >= nb || a[i] <= b[j]);
            out[t] = takeA ? a[i++] : b[j++];
        }
    }
    __syncwarp();
}

// Copies up to `need` ids of sorted block b whose in-block offset lies in
// [o1, o2), in ascending id order.  Returns the count.
__device__ __forceinline__ int load_partial(const DevIndex& ix, int64_t b, int o1, int o2,
                                            uint32_t* dst, int need) {
    const unsigned lane = lane_id();
    int cnt = 0;
    for (int base = 0; base < kBlk && cnt < need; base += 32) {
        int t = base + (int)lane;
        uint32_t id = ix.sblk[b * kBlk + t];
        int off = ix.soff[b * kBlk + t];
        bool keep = id != kInf && off >= o1 && off < o2;
        unsigned m = __ballot_sync(0xffffffffu, keep);
        int r = cnt + __popc(m & lanemask_lt());
        if (keep && r < need) dst[r] = id;
        cnt += __popc(m);
    }
    __syncwarp();
    return cnt < need ? cnt : need;
}

// Copies up to `need` leading valid ids of a sorted list.
__device__ __forceinline__ int load_list(const uint32_t* __restrict__ list, int len, uint32_t* dst,
                                         int need) {
    const unsigned lane = lane_id();
    int n = need < len ? need : len;
    int cnt = 0;
    for (int base = 0; base < n; base += 32) {
        int t = base + (int)lane;
        uint32_t id = t < n ? list[t] : kInf;
        if (t < n) dst[t] = id;
        cnt += __popc(__ballot_sync(0xffffffffu, t < n && id != kInf));
    }
    __syncwarp();
    return cnt;
}

// In-place removal of adjacent duplicates from a[0..n); returns new length.
__device__ __forceinline__ int warp_dedupe(const uint32_t* a, int n, uint32_t* out) {
    const unsigned lane = lane_id();
    int cnt = 0;
    for (int base = 0; base < n; base += 32) {
        int t = base + (int)lane;
        bool keep = t < n && (t == 0 || a[t] != a[t - 1]);
        unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) out[cnt + __popc(m & lanemask_lt())] = a[t];
        cnt += __popc(m);
    }
    __syncwarp();
    return cnt;
}

// The `need` smallest ids of sorted positions [lo, hi) into S.src[0].
__device__ int smallest_ids(const DevIndex& ix, int64_t lo, int64_t hi, int need, QWarp& S) {
    const int64_t bl0 = lo / kBlk, bh0 = (hi - 1) / kBlk;
    if (bl0 == bh0) return load_partial(ix, bl0, (int)(lo - bl0 * kBlk), (int)(hi - bl0 * kBlk), S.src[0], need);
    int c0 = 0, c1 = 0, c2 = 0, c3 = 0;
    int64_t bl = bl0, br = bh0 + 1;  // full blocks [bl, br)
    if (lo % kBlk) {
        c0 = load_partial(ix, bl0, (int)(lo % kBlk), kBlk, S.src[0], need);
        bl = bl0 + 1;
    }
    if (hi != ix.N && (hi % kBlk)) {
        c3 = load_partial(ix, bh0, 0, (int)(hi % kBlk), S.src[3], need);
        br = bh0;
    }
    if (br > bl) {
        int64_t span = br - bl;
        int j = 63 - __clzll((long long)span);
        const uint32_t* l1;
        const uint32_t* l2;
        int len;
        if (j == 0) {
            l1 = ix.sblk + bl * kBlk;
            l2 = ix.sblk + (br - 1) * kBlk;
            len = kBlk;
        } else {
            size_t lb = (size_t)(j - 1) * (size_t)ix.st_stride * (size_t)ix.K;
            l1 = ix.st + lb + (size_t)bl * ix.K;
            l2 = ix.st + lb + (size_t)(br - (1ll << j)) * ix.K;
            len = ix.K;
        }
        c1 = load_list(l1, len, S.src[1], need);
        if (span != (1ll << j)) c2 = load_list(l2, len, S.src[2], need);
    }
    // X = dedupe(merge(src1, src2)) in m2, Y = merge(src0, src3) in m1, M = merge(X, Y) in src0
    int cx;
    if (c2) {
        warp_merge(S.src[1], c1, S.src[2], c2, S.m1, c1 + c2);
        cx = warp_dedupe(S.m1, c1 + c2, S.m2);
    } else {
        for (int t = (int)lane_id(); t < c1; t += 32) S.m2[t] = S.src[1][t];
        __syncwarp();
        cx = c1;
    }
    if (cx > need) cx = need;
    int cy = c0 + c3 < need ? c0 + c3 : need;
    warp_merge(S.src[0], c0, S.src[3], c3, S.m1, cy);
    int cm = cx + cy < need ? cx + cy : need;
    warp_merge(S.m2, cx, S.m1, cy, S.src[0], cm);
    return cm;
}

// ---- one query, whole warp ----

__device__ void topk_one(const DevIndex& ix, QWarp& S, const uint8_t* qrow, const RowFmt& qf,
                         int64_t P0, int64_t P1, int k, int32_t* __restrict__ oid,
                         uint8_t* __restrict__ olcp) {
    const unsigned lane = lane_id();
    const int64_t N = ix.N;
    for (int w = (int)lane; w < ix.W; w += 32) S.q[w] = pack_word(qrow, w, qf);
    __syncwarp();
    // 2. lower bound inside the equal-head range, then both neighbours' LCPs
    int64_t lo = P0, hi = P1;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        int l;
        if (warp_cmp_row(ix.rows + mid * ix.W, S.q, ix, &l) < 0) lo = mid + 1;
        else hi = mid;
    }
    const int64_t p = lo;
    int lL = -1, lR = -1;
    if (p > 0) warp_cmp_row(ix.rows + (p - 1) * ix.W, S.q, ix, &lL);
    if (p < N) warp_cmp_row(ix.rows + p * ix.W, S.q, ix, &lR);
    // 3. expansion
    int nL = 0, nR = 0, dstar = 0;
    const int64_t availL = p, availR = N - p;
    for (;;) {
        int bL = nL < availL ? (nL == 0 ? lL : (int)S.llam[nL - 1]) : -1;
        int bR = nR < availR ? (nR == 0 ? lR : (int)S.rlam[nR - 1]) : -1;
        int F = bL > bR ? bL : bR;
        if (nL + nR >= k) {
            int v = kth_largest(S.llam, nL, S.rlam, nR, k);
            if (v >= F) {
                dstar = v;
                break;
            }
        }
        if (F < 0) {
            dstar = 0;  // all N < k items loaded
            break;
        }
        if (bL >= bR) {
            if (nL + 32 > kSide) {
                flag_status(ix.status, DEV_BAD);
                break;
            }
            int64_t x = p - 1 - nL - (int64_t)lane;
            bool ok = (int64_t)nL + lane < availL;
            int h = 255;
            uint32_t id = 0;
            if (ok) {
                h = (nL == 0 && lane == 0) ? lL : (int)ix.H[x + 1];
                id = (uint32_t)ix.ids[x];
            }
            if (nL > 0) h = min(h, (int)S.llam[nL - 1]);
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, h, o);
                if (lane >= (unsigned)o) h = min(h, y);
            }
            if (ok) {
                S.lid[nL + lane] = id;
                S.llam[nL + lane] = (uint8_t)h;
            }
            int64_t got = availL - nL < 32 ? availL - nL : 32;
            __syncwarp();
            nL += (int)got;
        } else {
            if (nR + 32 > kSide) {
                flag_status(ix.status, DEV_BAD);
                break;
            }
            int64_t x = p + nR + (int64_t)lane;
            bool ok = (int64_t)nR + lane < availR;
            int h = 255;
            uint32_t id = 0;
            if (ok) {
                h = (nR == 0 && lane == 0) ? lR : (int)ix.H[x];
                id = (uint32_t)ix.ids[x];
            }
            if (nR > 0) h = min(h, (int)S.rlam[nR - 1]);
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, h, o);
                if (lane >= (unsigned)o) h = min(h, y);
            }
            if (ok) {
                S.rid[nR + lane] = id;
                S.rlam[nR + lane] = (uint8_t)h;
            }
            int64_t got = availR - nR < 32 ? availR - nR : 32;
            __syncwarp();
            nR += (int)got;
        }
    }
    // A = loaded items with LCP > d*; interval of level d*
    const int aL = count_ge(S.llam, nL, dstar + 1);
    const int aR = count_ge(S.rlam, nR, dstar + 1);
    const int nA = aL + aR;
    int64_t lov, hiv;
    if (dstar == 0) {
        lov = 0;
        hiv = N;
    } else {
        int vL = count_ge(S.llam, nL, dstar);
        int vR = count_ge(S.rlam, nR, dstar);
        if (vL < nL || nL == availL) lov = p - vL;
        else {
            int64_t x = prev_less(ix, p - nL, dstar);
            lov = x < 0 ? 0 : x;
        }
        if (vR < nR || nR == availR) hiv = p + vR;
        else hiv = next_less(ix, p + nR, dstar);
    }
    const int64_t nT = (hiv - lov) - nA;
    int kp = k - nA;
    if ((int64_t)kp > nT) kp = (int)nT;
    // 4. tie fill: first kp ids of the level-d* interval outside A
    int ntake = 0;
    if (kp > 0) {
        int need = nA + kp;
        int cm = smallest_ids(ix, lov, hiv, need, S);
        const int64_t loc = p - aL, hic = p + aR;
        for (int base = 0; base < cm && ntake < kp; base += 32) {
            int t = base + (int)lane;
            uint32_t id = t < cm ? S.src[0][t] : kInf;
            bool keep = false;
            if (t < cm) {
                int64_t ps = ix.pos[id];
                keep = ps < loc || ps >= hic;
            }
            unsigned m = __ballot_sync(0xffffffffu, keep);
            int r = ntake + __popc(m & lanemask_lt());
            if (keep && r < kp) S.m1[r] = id;
            ntake += __popc(m);
        }
        if (ntake > kp) ntake = kp;
        __syncwarp();
    }
    // 5. sort A by (LCP desc, id asc)
    int P = 1;
    while (P < nA) P <<= 1;
    for (int t = (int)lane; t < P; t += 32) {
        uint64_t key = ~0ull;
        if (t < aL) key = ((uint64_t)(255 - S.llam[t]) << 32) | S.lid[t];
        else if (t < nA) key = ((uint64_t)(255 - S.rlam[t - aL]) << 32) | S.rid[t - aL];
        S.akey[t] = key;
    }
    __syncwarp();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = (int)lane; t < P; t += 32) {
                int u = t ^ stride;
                if (u > t) {
                    uint64_t a = S.akey[t], b = S.akey[u];
                    bool up = (t & size) == 0;
                    if ((a > b) == up) {
                        S.akey[t] = b;
                        S.akey[u] = a;
                    }
                }
            }
            __syncwarp();
        }
    }
    for (int r = (int)lane; r < k; r += 32) {
        int32_t id = -1;
        uint8_t l = 0;
        if (r < nA) {
            uint64_t key = S.akey[r];
            id = (int32_t)(uint32_t)key;
            l = (uint8_t)(255 - (int)(key >> 32));
        } else if (r < nA + ntake) {
            id = (int32_t)S.m1[r - nA];
            l = (uint8_t)dstar;
        }
        oid[r] = id;
        olcp[r] = l;
    }
    __syncwarp();
}

__global__ void __launch_bounds__(kSearchWarps * 32) k_topk_search(DevIndex ix,
                                                                   const uint8_t* __restrict__ queries,
                                                                   RowFmt qf, int64_t Q, int k,
                                                                   int32_t* __restrict__ out_ids,
                                                                   uint8_t* __restrict__ out_lcp) {
    __shared__ QWarp sm[kSearchWarps];
    const int warp = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    QWarp& S = sm[warp];
    const int64_t wq0 = ((int64_t)blockIdx.x * kSearchWarps + warp) * 32;
    if (wq0 >= Q) return;
    // 1. lane-per-query search on head
    const int64_t myq = wq0 + lane;
    const bool has = myq < Q;
    uint64_t q0 = has ? pack_word(row_of(queries, myq, qf), 0, qf) : 0;
    int64_t lo = 0, hi = ix.N;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (ix.head[mid] < q0) lo = mid + 1;
        else hi = mid;
    }
    const int64_t p0 = lo;
    hi = ix.N;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (ix.head[mid] <= q0) lo = mid + 1;
        else hi = mid;
    }
    const int64_t p1 = lo;
    for (int j = 0; j < 32; ++j) {
        const int64_t qi = wq0 + j;
        if (qi >= Q) break;
        const int64_t P0 = __shfl_sync(0xffffffffu, p0, j);
        const int64_t P1 = __shfl_sync(0xffffffffu, p1, j);
        topk_one(ix, S, row_of(queries, qi, qf), qf, P0, P1, k, out_ids + qi * k, out_lcp + qi * k);
    }
}

}  // namespace lcpk

namespace lcph {
using namespace lcpk;

int topk_batch_device(lcp_index_s* x, const void* d_queries, int64_t Q, int k, int32_t* out_ids,
                      uint8_t* out_lcp, cudaStream_t s) {
    if (Q <= 0) return LCP_OK;
    if (x->N == 0) {
        LCP_CUDA_TRY(cudaMemsetAsync(out_ids, 0xFF, sizeof(int32_t) * (size_t)Q * k, s));
        LCP_CUDA_TRY(cudaMemsetAsync(out_lcp, 0, (size_t)Q * k, s));
        return LCP_OK;
    }
    DevIndex ix = dev_view(x);
    RowFmt qf = make_fmt(x->tb, x->L, d_queries);
    int64_t warps = (Q + 31) / 32;
    unsigned grid = (unsigned)((warps + kSearchWarps - 1) / kSearchWarps);
    LCP_LAUNCH(k_topk_search, grid, kSearchWarps * 32, 0, s, ix,
               reinterpret_cast<const uint8_t*>(d_queries), qf, Q, k, out_ids, out_lcp);
    return LCP_OK;
}

}  // namespace lcph
