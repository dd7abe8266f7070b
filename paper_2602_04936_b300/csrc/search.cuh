// Warp-level building blocks shared by the indexed search and the build of
// its tie lists: shared-memory layout of one query's work area, warp sorts
// and merges, min-tree walks over H, and the "k smallest ids of a sorted
// position range" routine over the sparse table.
#pragma once

#include "index.cuh"

namespace lcpk {

constexpr int kSearchWarps = 4;
constexpr int kMaxW = 64;
constexpr int kKMax = LCP_INDEX_MAX_K;
constexpr int kSide = kKMax + 64;  // loaded items per side stay below k + 32

// Position record of one query (insertion point p, LCPs with rows p-1 and
// p, first token), written by the locate kernels.
struct alignas(16) QLoc {
    int64_t p;
    int16_t lL, lR;
    int32_t tok0;
};

struct alignas(16) QWarp {
    uint32_t src[4][kKMax];
    uint32_t m1[2 * kKMax];
    uint8_t llam[kSide];
    uint8_t rlam[kSide];
};

// The expansion's work area (a subset of QWarp): the loaded items' LCPs per
// side (their ids are read from the index when A is written).
struct alignas(16) AWarp {
    uint8_t llam[kSide];
    uint8_t rlam[kSide];
};

// The tie fill's work area (a subset of QWarp).
struct alignas(16) FWarp {
    uint32_t src[4][kKMax];
    uint32_t m1[2 * kKMax];
};

// ---------------------------------------------------------------------------
// sort keys: (255 - lcp) above the id, so ascending key = (lcp desc, id asc)
// ---------------------------------------------------------------------------
template <typename KT>
struct Key;
template <>
struct Key<uint32_t> {  // ids < 2^24
    static constexpr int kIdBits = 24;
};
template <>
struct Key<uint64_t> {
    static constexpr int kIdBits = 32;
};

template <typename KT>
__device__ __forceinline__ KT make_key(int lam, uint32_t id) {
    return ((KT)(255 - lam) << Key<KT>::kIdBits) | (KT)id;
}
template <typename KT>
__device__ __forceinline__ uint32_t key_id(KT k) {
    return (uint32_t)(k & (((KT)1 << Key<KT>::kIdBits) - 1));
}
template <typename KT>
__device__ __forceinline__ int key_lam(KT k) {
    return 255 - (int)(k >> Key<KT>::kIdBits);
}

// Ascending bitonic sort of 32*E keys held E per lane (lane l holds elements
// l*E .. l*E+E-1), entirely in registers.
template <int E, typename KT>
__device__ __forceinline__ void warp_bitonic(KT (&v)[E]) {
    const int lane = (int)lane_id();
#pragma unroll
    for (int size = 2; size <= 32 * E; size <<= 1) {
#pragma unroll
        for (int j = size >> 1; j > 0; j >>= 1) {
            if (j >= E) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int idx = lane * E + e;
                    KT o = __shfl_xor_sync(0xffffffffu, v[e], j / E);
                    const bool up = (idx & size) == 0;
                    const bool lower = (idx & j) == 0;
                    KT mn = v[e] < o ? v[e] : o;
                    KT mx = v[e] < o ? o : v[e];
                    v[e] = (lower == up) ? mn : mx;
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int pe = e ^ j;
                    if (pe > e) {
                        const bool up = ((lane * E + e) & size) == 0;
                        KT a = v[e], b = v[pe];
                        if ((a > b) == up) {
                            v[e] = b;
                            v[pe] = a;
                        }
                    }
                }
            }
        }
    }
}

// A of at most 32 items (left item i at position p-1-i, right item i at p+i;
// their ids read from the index): lane i holds item i and places it at its rank,
// the number of items whose key is smaller (keys are distinct: ids differ),
// found with nA broadcasts -- fewer instructions than a 32-key bitonic
// network whenever A is small, which it usually is.
template <typename KT, typename WA>
__device__ __forceinline__ void rank_and_write_A(const WA& S, const int32_t* __restrict__ ids, int p, int aL, int nA,
                                                 int32_t* __restrict__ oid,
                                                 uint8_t* __restrict__ olcp) {
    const int lane = (int)lane_id();
    KT key = ~(KT)0;
    if (lane < aL) key = make_key<KT>(S.llam[lane], (uint32_t)ids[p - 1 - lane]);
    else if (lane < nA) key = make_key<KT>(S.rlam[lane - aL], (uint32_t)ids[p + lane - aL]);
    int rank = 0;
    for (int j = 0; j < nA; j += 4) {  // four independent broadcasts per step
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const KT o = __shfl_sync(0xffffffffu, key, (j + u) & 31);
            rank += (j + u < nA) && o < key;
        }
    }
    if (lane < nA) {
        __stcs(oid + rank, (int)key_id<KT>(key));
        __stcs(reinterpret_cast<char*>(olcp) + rank, (char)key_lam<KT>(key));
    }
}

// Sorts A (left items [0, aL), right items [0, nA - aL)) and writes the
// first nA output slots.
template <int E, typename KT, typename WA>
__device__ __forceinline__ void sort_and_write_A(const WA& S, const int32_t* __restrict__ ids, int p, int aL, int nA,
                                                 int32_t* __restrict__ oid,
                                                 uint8_t* __restrict__ olcp) {
    const int lane = (int)lane_id();
    KT v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int idx = lane * E + e;
        KT key = ~(KT)0;
        if (idx < aL) key = make_key<KT>(S.llam[idx], (uint32_t)ids[p - 1 - idx]);
        else if (idx < nA) key = make_key<KT>(S.rlam[idx - aL], (uint32_t)ids[p + idx - aL]);
        v[e] = key;
    }
    warp_bitonic<E, KT>(v);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int idx = lane * E + e;
        if (idx < nA) {
            __stcs(oid + idx, (int)key_id<KT>(v[e]));  // streaming: results are not re-read
            __stcs(reinterpret_cast<char*>(olcp) + idx, (char)key_lam<KT>(v[e]));
        }
    }
}

// ---- warp-wide comparison against the query held in shared memory ----

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

// LCPs of q with rows p-1 and p (-1 where the row does not exist); both rows'
// words are loaded before either is compared.
__device__ __forceinline__ void warp_lcp_neighbours(const DevIndex& ix, int64_t p, const uint64_t* q,
                                                    int* lL, int* lR) {
    const unsigned lane = lane_id();
    const bool hasL = p > 0, hasR = p < ix.N;
    int fl = -1, fr = -1;  // first differing word (or -1 if none yet)
    for (int w0 = 0; w0 < ix.W && (fl < 0 || fr < 0); w0 += 32) {
        const int w = w0 + (int)lane;
        const bool in = w < ix.W;
        const uint64_t qw = in ? q[w] : 0;
        const uint64_t a = (in && hasL) ? ix.rows[(p - 1) * ix.W + w] : qw;
        const uint64_t b = (in && hasR) ? ix.rows[p * ix.W + w] : qw;
        const unsigned ml = __ballot_sync(0xffffffffu, a != qw);
        const unsigned mr = __ballot_sync(0xffffffffu, b != qw);
        if (fl < 0 && ml) {
            const int f = __ffs(ml) - 1;
            const uint64_t x = __shfl_sync(0xffffffffu, a ^ qw, f);
            fl = (w0 + f) * ix.tpw + (__clzll((long long)x) / ix.bits);
        }
        if (fr < 0 && mr) {
            const int f = __ffs(mr) - 1;
            const uint64_t x = __shfl_sync(0xffffffffu, b ^ qw, f);
            fr = (w0 + f) * ix.tpw + (__clzll((long long)x) / ix.bits);
        }
    }
    *lL = hasL ? (fl < 0 || fl > ix.L ? ix.L : fl) : -1;
    *lR = hasR ? (fr < 0 || fr > ix.L ? ix.L : fr) : -1;
}

// ---- min tree over H: interval ends at level d, both sides interleaved ----

__device__ __forceinline__ const uint8_t* hlevel(const DevIndex& ix, int lev) {
    return lev == 0 ? ix.H : ix.hmin + ix.hoff[lev];
}

// State of one side's search: climbing until a group holding an H < d is
// found, then descending to level 0.
struct BoundSearch {
    int idx;
    int lev;
    int phase;  // 0 climb, 1 descend, 2 done
    int result;
};

// Left side: largest x <= from with H[x] < d (or -1).  Right side: smallest
// x >= from with H[x] < d (or N).  `need*` = 0 skips a side.  Positions are
// 32-bit (an index holds fewer than 2^30 rows).
__device__ __forceinline__ void find_bounds(const DevIndex& ix, int fromL, bool needL, int fromR, bool needR,
                            int d, int* outL, int* outR) {
    const unsigned lane = lane_id();
    const int N = (int)ix.N;
    BoundSearch s[2];
    s[0] = {fromL, 0, needL ? 0 : 2, -1};
    s[1] = {fromR, 0, needR ? 0 : 2, N};
    if (needR && fromR >= N) s[1].phase = 2;
    if (needL && fromL < 0) s[0].phase = 2;
    while (s[0].phase != 2 || s[1].phase != 2) {
        uint8_t val[2];
        int e[2], g0[2];
        bool inr[2];
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            BoundSearch& b = s[side];
            inr[side] = false;
            val[side] = 255;
            if (b.phase == 2) continue;
            const int lev = b.phase == 0 ? b.lev : b.lev - 1;
            const uint8_t* arr = hlevel(ix, lev);
            const int len = (int)ix.hlen[lev];
            g0[side] = b.phase == 0 ? ((b.idx >> 5) << 5) : (b.idx << 5);
            e[side] = g0[side] + (int)lane;
            bool ok = e[side] < len;
            if (b.phase == 0) ok = ok && (side == 0 ? e[side] <= b.idx : e[side] >= b.idx);
            inr[side] = ok;
            if (ok) val[side] = arr[e[side]];
        }
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            BoundSearch& b = s[side];
            if (b.phase == 2) continue;
            unsigned m = __ballot_sync(0xffffffffu, inr[side] && (int)val[side] < d);
            if (b.phase == 0) {
                if (m) {
                    b.idx = g0[side] + (side == 0 ? 31 - __clz(m) : __ffs(m) - 1);
                    if (b.lev == 0) {
                        b.result = b.idx;
                        b.phase = 2;
                    } else {
                        b.phase = 1;
                    }
                } else if (b.lev == ix.hlev) {
                    b.phase = 2;
                } else {
                    b.idx = side == 0 ? (b.idx >> 5) - 1 : (b.idx >> 5) + 1;
                    ++b.lev;
                    if (b.idx < 0 || b.idx >= (int)ix.hlen[b.lev]) b.phase = 2;
                }
            } else {
                --b.lev;
                if (!m) {  // impossible in a consistent tree
                    flag_status(ix.status, DEV_BAD);
                    b.phase = 2;
                    continue;
                }
                b.idx = g0[side] + (side == 0 ? 31 - __clz(m) : __ffs(m) - 1);
                if (b.lev == 0) {
                    b.result = b.idx;
                    b.phase = 2;
                }
            }
        }
    }
    *outL = s[0].result;
    *outR = s[1].result;
}

// The run of sorted rows whose first d <= tpw tokens equal q's, where only
// word 0 (the head array) decides: `key` = a row of the run's word 0 masked
// to its first d tokens.  Left: the first x in [b0, from) with head[x] in
// the run (it ends at `from`); right: the first x in [from, b1) past it.
// 32-ary searches (lane l probes the l-th of 32 evenly spaced positions,
// a ballot finds the first that satisfies), both sides' loads in flight
// together; [b0, b1) is the depth-1 bucket holding the run.
__device__ __forceinline__ void head_bounds(const DevIndex& ix, int b0, int b1, int fromL, int fromR,
                                            uint64_t key, uint64_t mask, bool needL, bool needR, int* outL,
                                            int* outR) {
    const int lane = (int)lane_id();
    int lo[2] = {b0, fromR}, hi[2] = {fromL, b1};
    bool done[2] = {!needL || b0 >= fromL, !needR || fromR >= b1};
    {  // galloping round (runs are usually far shorter than the bucket): lane i
       // probes 2^i positions out from the known part, bracketing each end
        uint64_t h[2] = {0ull, 0ull};
        int x[2];
        x[0] = max(fromL - (1 << lane), b0);
        { const long long xr = (long long)fromR + (1ll << lane) - 1; x[1] = (int)(xr < (long long)b1 - 1 ? xr : (long long)b1 - 1); }
#pragma unroll
        for (int sd = 0; sd < 2; ++sd)
            if (!done[sd]) h[sd] = ix.head[x[sd]];
        if (!done[0]) {  // rows at and right of the answer satisfy: the first lane that fails
            const unsigned m = __ballot_sync(0xffffffffu, (h[0] & mask) >= key);
            const unsigned fail = ~m;
            const int j = __ffs(fail) - 1;  // lanes past x = b0 repeat b0's answer
            if (!fail) {
                hi[0] = b0;
                done[0] = true;
            } else {
                const int xj = __shfl_sync(0xffffffffu, x[0], j);
                const int xp = j == 0 ? fromL : __shfl_sync(0xffffffffu, x[0], j - 1 < 0 ? 0 : j - 1);
                lo[0] = xj + 1;
                hi[0] = xp;
                if (lo[0] >= hi[0]) done[0] = true;
            }
        }
        if (!done[1]) {  // the first row past the run: the first lane that passes
            const unsigned m = __ballot_sync(0xffffffffu, (h[1] & mask) > key);
            if (!m) {
                hi[1] = b1;
                done[1] = true;
            } else {
                const int j = __ffs(m) - 1;
                const int xj = __shfl_sync(0xffffffffu, x[1], j);
                const int xp = j == 0 ? fromR - 1 : __shfl_sync(0xffffffffu, x[1], j - 1 < 0 ? 0 : j - 1);
                lo[1] = xp + 1;
                hi[1] = xj;
                if (lo[1] >= hi[1]) done[1] = true;
            }
        }
    }
    while (!(done[0] && done[1])) {  // warp-uniform
        int st[2], x[2];
        uint64_t h[2] = {0ull, 0ull};
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
            st[sd] = (hi[sd] - lo[sd] + 31) >> 5;
            x[sd] = min(lo[sd] + (lane + 1) * st[sd] - 1, hi[sd] - 1);
            if (!done[sd]) h[sd] = ix.head[x[sd]];
        }
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
            if (done[sd]) continue;
            const uint64_t v = h[sd] & mask;
            const unsigned m = __ballot_sync(0xffffffffu, sd == 0 ? v >= key : v > key);
            if (!m) {  // none up to hi - 1: the answer is hi
                done[sd] = true;
                continue;
            }
            const int f = __ffs(m) - 1;
            const int nlo = f == 0 ? lo[sd] : min(lo[sd] + f * st[sd] - 1, hi[sd] - 1) + 1;
            const int nhi = min(lo[sd] + (f + 1) * st[sd] - 1, hi[sd] - 1);  // satisfies
            lo[sd] = nlo;
            hi[sd] = nhi;
            if (nlo >= nhi) done[sd] = true;
        }
    }
    *outL = hi[0];
    *outR = hi[1];
}

// Minimum of H over positions [a, b] (inclusive), walking the min tree
// bottom-up: partial groups at both ends at each level, full groups above.
__device__ __forceinline__ int range_min_H(const DevIndex& ix, int64_t a, int64_t b) {
    const unsigned lane = lane_id();
    unsigned res = 255;
    int lev = 0;
    while (a <= b) {
        const uint8_t* arr = hlevel(ix, lev);
        const int64_t ga = a >> 5, gb = b >> 5;
        if (ga == gb) {
            const int64_t e = (ga << 5) + lane;
            const unsigned v = (e >= a && e <= b) ? arr[e] : 255u;
            res = min(res, __reduce_min_sync(0xffffffffu, v));
            break;
        }
        const int64_t ea = (ga << 5) + lane, eb = (gb << 5) + lane;
        const unsigned v1 = ea >= a ? arr[ea] : 255u;  // group ga is full (it is not the last)
        const unsigned v2 = eb <= b ? arr[eb] : 255u;
        res = min(res, __reduce_min_sync(0xffffffffu, min(v1, v2)));
        a = ga + 1;
        b = gb - 1;
        if (++lev > ix.hlev) break;
    }
    return (int)res;
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

// Ballot-compacts up to 4 candidates per lane (element t = lane + 32*e, in
// order) that pass `keep` into dst; at most `cap` are written.  Returns the
// number kept (capped).
__device__ __forceinline__ int compact4(const uint32_t (&v)[4], const bool (&keep)[4], uint32_t* dst,
                                        int cap) {
    const unsigned lt = lanemask_lt();
    int cnt = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        unsigned m = __ballot_sync(0xffffffffu, keep[e]);
        int r = cnt + __popc(m & lt);
        if (keep[e] && r < cap) dst[r] = v[e];
        cnt += __popc(m);
    }
    return cnt < cap ? cnt : cap;
}

// The `need` smallest ids of sorted positions [lo, hi) into S.src[0]
// (need <= kKMax).  Returns how many there are (min(need, hi - lo)).
template <typename WA>  // QWarp or FWarp: uses src and m1
__device__ __forceinline__ int smallest_ids(const DevIndex& ix, int64_t lo, int64_t hi, int need, WA& S) {
    const unsigned lane = lane_id();
    const int64_t bl0 = lo / kBlk, bh0 = (hi - 1) / kBlk;
    // source descriptors
    int64_t pb[2] = {-1, -1};  // partial blocks (left, right)
    int po1[2] = {0, 0}, po2[2] = {0, 0};
    const uint32_t* lst[2] = {nullptr, nullptr};
    int llen = 0;
    if (bl0 == bh0) {
        pb[0] = bl0;
        po1[0] = (int)(lo - bl0 * kBlk);
        po2[0] = (int)(hi - bl0 * kBlk);
    } else {
        int64_t bl = bl0, br = bh0 + 1;
        if (lo % kBlk) {
            pb[0] = bl0;
            po1[0] = (int)(lo % kBlk);
            po2[0] = kBlk;
            bl = bl0 + 1;
        }
        if (hi != ix.N && (hi % kBlk)) {
            pb[1] = bh0;
            po1[1] = 0;
            po2[1] = (int)(hi % kBlk);
            br = bh0;
        }
        if (br > bl) {
            const int64_t span = br - bl;
            const int j = 63 - __clzll((long long)span);
            if (j == 0) {
                lst[0] = ix.sblk + bl * kBlk;
                llen = kBlk;
            } else {
                const size_t lb = (size_t)(j - 1) * (size_t)ix.st_stride * (size_t)ix.K;
                lst[0] = ix.st + lb + (size_t)bl * ix.K;
                if (span != (1ll << j)) lst[1] = ix.st + lb + (size_t)(br - (1ll << j)) * ix.K;
                llen = ix.K;
            }
        }
    }
    // issue every load before consuming any (independent, all in flight)
    uint32_t pv[2][4], lv[2][4];
    uint8_t po[2][4];
    const int ln = need < llen ? need : llen;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int t = (int)lane + 32 * e;
            pv[s][e] = kInf;
            po[s][e] = 0;
            lv[s][e] = kInf;
            if (pb[s] >= 0) {
                pv[s][e] = ix.sblk[pb[s] * kBlk + t];
                po[s][e] = ix.soff[pb[s] * kBlk + t];
            }
            if (lst[s] && t < ln) lv[s][e] = lst[s][t];
        }
    }
    int c[4];  // src0 = left partial, src1/2 = lists, src3 = right partial
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        bool keep[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
            keep[e] = pv[s][e] != kInf && (int)po[s][e] >= po1[s] && (int)po[s][e] < po2[s];
        c[s == 0 ? 0 : 3] = pb[s] >= 0 ? compact4(pv[s], keep, S.src[s == 0 ? 0 : 3], need) : 0;
        bool vk[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) vk[e] = lv[s][e] != kInf;
        c[1 + s] = lst[s] ? compact4(lv[s], vk, S.src[1 + s], need) : 0;
    }
    __syncwarp();
    if (c[1] + c[2] == 0 && c[3] == 0) return c[0];
    if (c[1] + c[2] == 0 && c[0] == 0) {
        for (int t = (int)lane; t < c[3]; t += 32) S.src[0][t] = S.src[3][t];
        __syncwarp();
        return c[3];
    }
    // X = dedupe(merge(src1, src2)) -> src1 ; Y = merge(src0, src3) -> src2 ; M -> src0
    int cx = c[1];
    if (c[2]) {
        warp_merge(S.src[1], c[1], S.src[2], c[2], S.m1, c[1] + c[2]);
        const unsigned lt = lanemask_lt();
        int cnt = 0;
        for (int base = 0; base < c[1] + c[2] && cnt < need; base += 32) {
            int t = base + (int)lane;
            bool keep = t < c[1] + c[2] && (t == 0 || S.m1[t] != S.m1[t - 1]);
            unsigned m = __ballot_sync(0xffffffffu, keep);
            int r = cnt + __popc(m & lt);
            if (keep && r < need) S.src[1][r] = S.m1[t];
            cnt += __popc(m);
        }
        __syncwarp();
        cx = cnt < need ? cnt : need;
    }
    const int cy = c[0] + c[3] < need ? c[0] + c[3] : need;
    warp_merge(S.src[0], c[0], S.src[3], c[3], S.src[2], cy);
    const int cm = cx + cy < need ? cx + cy : need;
    warp_merge(S.src[1], cx, S.src[2], cy, S.src[0], cm);
    return cm;
}

}  // namespace lcpk

namespace lcpk {

// ---- persistent worker fed by a work queue (queue.cu holds the host side) ----

// One request.  The host fills it in pinned memory and copies it, with the
// request's task records, to device memory on a copy stream; the new task
// count is copied after them on the same stream, so a worker that sees the
// count also sees the records.  The worker reads only device memory.
struct QReq {
    DevIndex ix;           // snapshot of the index at submission
    const uint8_t* queries;
    RowFmt qf;
    int32_t k;
    int32_t ntasks;        // tasks the request was cut into
    int32_t* out_ids;
    uint8_t* out_lcp;
    uint64_t ticket;
};

// One task: queries [q0, q1) of the request in slot `slot`.
struct QTask {
    int64_t q0, q1;
    int32_t slot;
    int32_t pad;
};

// Control words in device memory, written by host copies.
struct QCtl {
    int64_t published;  // tasks published so far
    int32_t stop;       // set at shutdown: idle warps exit at once
    int32_t pad;
};

struct QueueArgs {
    const QCtl* ctl;       // device
    const QReq* reqs;      // device [rcap]
    const QTask* tasks;    // device [tcap]
    uint64_t* done;        // mapped host memory [rcap]: ticket of the last completed request per slot
    int64_t* claimed;        // device: next task id to claim
    int64_t* min_abandoned;  // device: smallest id given up unpublished in this launch
    unsigned* exited;        // device: warps of this launch that have left
    int64_t* taken;          // device: [tcap] largest id taken from each ring slot (-1 at start)
    int32_t* done_count;   // device: [rcap] finished tasks of the slot's request
    int rcap, tcap;
    long long idle_ns;     // a warp that finds no work for this long exits
    int* status;           // device status word
};

}  // namespace lcpk

namespace lcph {
// Launches the persistent worker (grid CTAs of kSearchWarps warps) on s.
void launch_queue_worker(const lcpk::QueueArgs& a, unsigned grid, cudaStream_t s);

// Locates every query of a batch into loc[Q]: warp per query (warp_mode 1),
// lane per query (0), or by batch size (-1).
void launch_locate(const lcpk::DevIndex& ix, const uint8_t* q, const lcpk::RowFmt& qf, int64_t Q,
                   lcpk::QLoc* loc, cudaStream_t s, int warp_mode = -1);

// Launch shape of the indexed search: the heuristic, and the process-wide
// table of autotuned shapes keyed by (log2 N, L, token bytes, log2 Q, k class).
SearchShape default_shape(int64_t Q);
SearchShape search_shape(const lcp_index_s* x, int64_t Q, int k);
void set_search_shape(const lcp_index_s* x, int64_t Q, int k, const SearchShape& sh);
}  // namespace lcph

