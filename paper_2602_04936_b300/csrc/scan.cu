// Full scan top-k: LCP of every query against all N rows (the paper's "full
// scan" baseline, Sec. 7), no index over the rows.
//
// Batches of more than kSelMaxQ queries:
//   k_pack_plane0   word 0 of every row, packed, into a plane of upper and
//                   lower halves (8 bytes a row: 16 MB at N=2M, so it stays
//                   in L2 while the query tiles stream over it); tiles of it
//                   reach shared memory by bulk copies (the TMA unit),
//                   double-buffered.
//   (batch order)   the queries sorted by their first word (one CTA up to
//                   4,096 queries, the radix sort above), so that a warp's 32
//                   queries are neighbours in word-0 order.
//   k_scan_partial  grid = (query tiles) x (N slices); a thread owns one query
//                   and logs the rows of its slice that can still be in its
//                   top k: rows arrive in increasing id, so once k are held
//                   only rows above a level `worst` can matter, i.e. rows whose
//                   word 0 lies in a prefix range [lo, hi] of q's.  The warp
//                   screens a row with one lane-parallel test against the
//                   union of its lanes' ranges (narrow: the queries are
//                   neighbours), and only rows inside it are tested by every
//                   lane; the exact LCP over later words is computed for rows
//                   inside a lane's own range.  When the log holds k + 64 rows
//                   it is cut back to k (rows above the k-th largest LCP, the
//                   earliest at it) and worst rises.  Levels with k rows at or
//                   above them are shared between a query's slices (an atomic
//                   maximum, read at every tile), seeded by a first pass over a
//                   sample of the rows.
//   k_scan_merge    keys (255 - LCP) << 32 | id are unique, so the k smallest
//                   over a query's slice logs are order independent: keys below
//                   the best shared level and, once k are held, above the k-th
//                   are dropped as they are read; the rest are sorted in shared
//                   memory.  Written to the query's own output row.
// Smaller batches take the threshold selection (scan_select.cu).
#include "scan.cuh"
#include "sort.cuh"

namespace lcpk {

constexpr int kScanTile = 1024;     // plane-0 words per shared-memory tile
constexpr int kScanStages = 3;      // tiles in the ring
constexpr int kScanAhead = 1;       // tiles in flight beyond the one screened
// With at least two spare buffers in the ring the buffer a copy refills was
// last read two tiles back, before the previous tile's wait barrier, so a
// tile needs no barrier of its own at its end.
constexpr bool kScanEndBarrier = kScanStages - kScanAhead < 2;
constexpr int kCompactBins = 16;    // levels above `worst` a log compaction counts in one pass
constexpr uint64_t kKeyInf = ~0ull;

// Packed word 0 of a row.  Aligned rows are read with one 8-byte load that
// asks L2 for a 64-byte fetch rather than the row's whole line.
__device__ __forceinline__ uint64_t row_word0(const uint8_t* row, const RowFmt& f) {
    if (f.aligned8) {
        unsigned long long x;
        asm("ld.global.nc.L2::64B.u64 %0, [%1];" : "=l"(x) : "l"(row));
        return msb_first(x, f.tb);
    }
    return pack_word(row, 0, f);
}

__global__ void k_pack_plane0(const uint8_t* __restrict__ tokens, RowFmt f, int64_t n,
                              uint32_t* __restrict__ plane_hi, uint32_t* __restrict__ plane_lo) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const uint64_t w = row_word0(row_of(tokens, i, f), f);
        plane_hi[i] = (uint32_t)(w >> 32);
        plane_lo[i] = (uint32_t)w;
    }
}

// Word-0 mask that tests "the first t tokens are equal" (t <= tpw).
__device__ __forceinline__ uint64_t prefix_mask(int t, int bits) {
    int b = t * bits;
    return b >= 64 ? ~0ull : (b == 0 ? 0ull : (~0ull << (64 - b)));
}

__global__ void __launch_bounds__(kScanPartialThreads, 2) k_scan_partial(const ScanArgs a) {
    __shared__ __align__(128) uint32_t tile_hi[kScanStages][kScanTile];  // plane tiles (upper halves),
    __shared__ __align__(128) uint32_t tile_lo[kScanStages][kScanTile];  // a ring of kScanStages
    __shared__ __align__(8) uint64_t tbar[kScanStages];                  // their bulk-copy barriers
    __shared__ uint16_t cbins[kCompactBins][kScanPartialThreads];
    const RowFmt& f = a.f;
    const int k = a.k;
    const unsigned lane = lane_id();
    const int64_t qs = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // position in the batch order
    const int64_t s0 = (int64_t)blockIdx.y * a.slice;
    const int64_t s1 = s0 + a.slice < a.N ? s0 + a.slice : a.N;
    const bool active = qs < a.Q;
    const int64_t qi = active ? (a.order ? (int64_t)a.order[qs] : qs) : 0;
    const uint8_t* qrow = active ? row_of(a.queries, qi, a.qf) : nullptr;
    const uint64_t q0 = active ? pack_word(qrow, 0, a.qf) : 0;
    // the thread's log: keys (255 - LCP) << 32 | id of the rows taken, in id
    // order (rows arrive in increasing id), at most cap of them
    uint64_t* log = a.lists + ((int64_t)blockIdx.y * a.Q + (active ? qs : 0)) * a.cap;
    int n = 0;
    // -1 until k rows are logged (every row is taken); then a level with k
    // rows of this slice, of smaller id, at or above it -- or, from the
    // floor, with k rows anywhere at or above it + 1 -- so that only rows of
    // LCP > worst can still matter: rows whose first worst + 1 tokens equal
    // q's, i.e. whose word 0 lies in [lo, hi] (all of word 0 equal once
    // worst + 1 >= tpw; deeper words then decide)
    int worst = -1;
    int lvl = 0;  // a level with k rows anywhere at or above it (0: none known)
    uint64_t T = 0, lo = 0, hi = ~0ull;
    auto set_range = [&]() {
        if (worst < 0) {
            lo = 0;
            hi = ~0ull;
            return;
        }
        const int b = (worst + 1) * f.bits;
        T = b >= 64 ? 1ull : (1ull << (64 - b));
        lo = q0 & ~(T - 1);
        hi = lo | (T - 1);
    };
    // Takes a shared level: k rows have LCP >= fl, so rows below it cannot
    // be in the answer.
    auto take_floor = [&](int fl) {
        if (fl <= lvl) return false;
        lvl = fl;
        if (fl - 1 <= worst) return false;
        worst = fl - 1;
        set_range();
        return true;
    };
    if (active && a.floor) take_floor((int)ld_relaxed(reinterpret_cast<const uint32_t*>(a.floor) + qs));
    set_range();
    auto lam_of = [](uint64_t e) { return 255 - (int)(e >> 32); };
    // Raises worst to the largest w with >= k logged rows of LCP >= w and
    // keeps the rows above w and the earliest (smallest-id) ones at w, k in
    // all.  A row dropped here, or refused later for LCP <= worst, has k
    // rows of smaller id and no smaller LCP: it is in no top k.
    uint16_t* hist = &cbins[0][threadIdx.x];  // this thread's level counts, stride kScanPartialThreads
    auto compact = [&]() {
        int w;
        if (worst < 0) {  // the first k rows (n == k): w = their smallest LCP, all kept
            w = 255;
            for (int i = 0; i < n; ++i) w = min(w, lam_of(log[i]));
        } else {
            // one pass: counts of the logged levels worst + 1 + j (bin kCompactBins - 1
            // open-ended; rows at or below worst, logged before a shared level
            // raised it, are not counted and are dropped below)
#pragma unroll
            for (int j = 0; j < kCompactBins; ++j) hist[j * kScanPartialThreads] = 0;
            for (int i = 0; i < n; ++i) {
                const int d = lam_of(log[i]) - worst - 1;
                if (d >= 0) ++hist[min(d, kCompactBins - 1) * kScanPartialThreads];
            }
            // the smallest w >= worst with fewer than k logged rows above it
            int above = 0;
            for (int j = 0; j < kCompactBins; ++j) above += hist[j * kScanPartialThreads];
            w = worst;
            for (int j = 0; j < kCompactBins - 1 && above >= k; ++j) {
                above -= hist[j * kScanPartialThreads];
                ++w;
            }
            if (above >= k) {  // beyond the bins (rare): count level by level
                for (;;) {
                    int c = 0;
                    for (int i = 0; i < n; ++i) c += lam_of(log[i]) > w;
                    if (c < k) break;
                    ++w;
                }
            }
        }
        int above = 0;
        int m = 0;
        if (worst >= 0 || n > k) {
            for (int i = 0; i < n; ++i) above += lam_of(log[i]) > w;
            int eq = k - above;
            for (int i = 0; i < n; ++i) {
                const uint64_t e = log[i];
                const int l = lam_of(e);
                if (l > w || (l == w && eq-- > 0)) log[m++] = e;
            }
        } else {
            m = n;
        }
        n = m;
        worst = w;
        set_range();
        if (w > lvl) {  // this slice alone has k rows at or above w: share it
            lvl = w;
            if (a.floor) atomicMax(a.floor + qs, w);
        }
    };
    auto row_at = [&](int64_t id, uint64_t r) {  // a row inside the thread's range
        int lam;
        const uint64_t x = r ^ q0;
        if (x) {
            lam = __clzll((long long)x) / f.bits;
        } else {
            lam = f.L;
            const uint8_t* row = row_of(a.tokens, id, f);
            for (int w = 1; w < f.W; ++w) {
                const uint64_t y = pack_word(row, w, f) ^ pack_word(qrow, w, a.qf);
                if (y) {
                    lam = w * f.tpw + (__clzll((long long)y) / f.bits);
                    break;
                }
            }
        }
        if (lam > f.L) lam = f.L;
        if (worst >= 0 && lam <= worst) return;
        log[n++] = ((uint64_t)(255 - lam) << 32) | (uint64_t)id;
        if (worst < 0 ? n == k : n == a.cap) compact();
    };
    // The warp's screen: the union of its lanes' ranges lies in [WL, WL +
    // span] on the upper halves of word 0.  The batch is ordered by the
    // queries' first words, so neighbouring lanes hold neighbouring ranges
    // and the union is narrow once the lanes' levels have risen: a lane tests
    // one row of each 32 against it, and only the rows inside are compared
    // by every lane with its own query.
    uint32_t WL = 0, span = 0;
    auto refresh = [&]() {
        WL = __reduce_min_sync(0xffffffffu, active ? (uint32_t)(lo >> 32) : 0xffffffffu);
        const uint32_t WH = __reduce_max_sync(0xffffffffu, active ? (uint32_t)(hi >> 32) : 0u);
        span = WH - WL;
    };
    const bool warp_any = __any_sync(0xffffffffu, active);
    refresh();
    // The plane tiles arrive by bulk copies (the TMA unit) into a ring of
    // kScanStages buffers: the next kScanAhead tiles are in flight while one
    // is screened.  Thread 0 issues and waits; every wait is bounded.
    if (threadIdx.x == 0) {
        for (int b = 0; b < kScanStages; ++b) mbar_init(&tbar[b], 1);
        fence_proxy_async_smem();
    }
    __syncthreads();
    auto issue = [&](int64_t t, int b) {  // thread 0: tile starting at row t into buffer b
        const int n = (int)(s1 - t < kScanTile ? s1 - t : kScanTile);
        const uint32_t bytes = (uint32_t)((n * 4 + 15) & ~15);  // the plane is padded to 16 bytes
        mbar_arrive_expect_tx(&tbar[b], 2 * bytes);
        bulk_g2s(&tile_hi[b][0], a.plane_hi + t, bytes, &tbar[b]);
        bulk_g2s(&tile_lo[b][0], a.plane_lo + t, bytes, &tbar[b]);
    };
    const int ntiles = s0 < s1 ? (int)((s1 - s0 + kScanTile - 1) / kScanTile) : 0;
    if (threadIdx.x == 0)
        for (int t = 0; t < kScanAhead && t < ntiles; ++t) issue(s0 + (int64_t)t * kScanTile, t);
    int it = 0;
    for (int64_t t0 = s0; t0 < s1; t0 += kScanTile, ++it) {
        const int tn = (int)(s1 - t0 < kScanTile ? s1 - t0 : kScanTile);
        const int buf = it % kScanStages;
        const uint32_t parity = (uint32_t)((it / kScanStages) & 1);
        // the buffer refilled here was last read by every thread before a
        // barrier they have all passed (the previous tile's wait barrier, or
        // its end barrier): those reads have returned their values, so the
        // copy cannot overtake them
        const int ahead = it + kScanAhead;
        if (threadIdx.x == 0 && ahead < ntiles) issue(s0 + (int64_t)ahead * kScanTile, ahead % kScanStages);
        // one thread waits for the tile (its acquire and the CTA barrier
        // make the copied words visible to all; many pollers would crowd
        // the shared-memory pipe the screen uses)
        const bool ok = threadIdx.x != 0 || mbar_wait(&tbar[buf], parity, kSpinLimit);
        if (__syncthreads_or(!ok)) {
            // the copy never completed: report it, let the copies in flight
            // land (bounded) before the CTA's shared memory is released
            if (threadIdx.x == 0) {
                flag_status(a.status, DEV_TIMEOUT);
                for (int t = it; t <= ahead && t < ntiles; ++t)
                    mbar_wait(&tbar[t % kScanStages], (uint32_t)((t / kScanStages) & 1), kSpinLimit);
            }
            __syncthreads();
            return;
        }
        if (!warp_any) {  // warp-uniform
            if (kScanEndBarrier) __syncthreads();
            continue;
        }
        if (a.floor) {  // levels other slices have shared since
            const bool up = active && take_floor((int)ld_relaxed(reinterpret_cast<const uint32_t*>(a.floor) + qs));
            if (__any_sync(0xffffffffu, up)) refresh();
        }
        for (int j0 = 0; j0 < tn; j0 += 32) {
            const int j = j0 + (int)lane;
            unsigned m = __ballot_sync(0xffffffffu, j < tn && tile_hi[buf][j] - WL <= span);
            bool moved = false;
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const uint64_t r = ((uint64_t)tile_hi[buf][j0 + b] << 32) | tile_lo[buf][j0 + b];
                if (active && (worst < 0 || (r ^ q0) < T)) {
                    const int w0 = worst;
                    row_at(t0 + j0 + b, r);
                    moved |= worst != w0;
                }
            }
            if (__any_sync(0xffffffffu, moved)) refresh();
        }
        if (kScanEndBarrier) __syncthreads();  // this buffer is refilled with the next tile
    }
    if (active) {
        if (n > k) compact();
        if (a.counts) a.counts[(int64_t)blockIdx.y * a.Q + qs] = n | (lvl << 16);
    }
}

// The k smallest keys over the S lists of batch position qs (counts[s][qs]
// = valid keys | level << 16, the level having k rows at or above it),
// sorted, written to the query's output row.  Keys below the highest such
// level, and -- once k keys are held -- keys above the k-th, cannot be in the
// answer and are dropped as they are read; the rest collect in shared memory,
// which is sorted (k kept) whenever it fills and at the end.  Keys are
// unique, so the result does not depend on the order of reading.  One CTA per
// batch position.
__global__ void __launch_bounds__(256) k_scan_merge(const uint64_t* __restrict__ lists,
                                                    const int32_t* __restrict__ counts, int cap, int64_t Q,
                                                    int S, int k, const int32_t* __restrict__ order,
                                                    int32_t* __restrict__ out_ids,
                                                    uint8_t* __restrict__ out_lcp) {
    extern __shared__ uint64_t keys[];           // kMergeCap
    __shared__ int32_t pre[kMergeMaxLists + 1];  // exclusive prefix of the lists' counts
    __shared__ int32_t wsum[8], wmax[8];
    __shared__ int used_sh;
    const int64_t qs = blockIdx.x;
    const int64_t qi = order ? (int64_t)order[qs] : qs;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int carry = 0, F = 0;
    for (int b0 = 0; b0 < S; b0 += 256) {
        const int s = b0 + tid;
        const int raw = s < S ? counts[(int64_t)s * Q + qs] : 0;
        const int c = raw & 0xffff;
        int x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const int lv = __reduce_max_sync(0xffffffffu, raw >> 16);
        if (lane == 31) wsum[warp] = x;
        if (lane == 0) wmax[warp] = lv;
        __syncthreads();
        int add = carry;
        for (int w = 0; w < warp; ++w) add += wsum[w];
        for (int w = 0; w < 8; ++w) F = max(F, wmax[w]);
        if (s < S) pre[s] = add + x - c;
        __syncthreads();
        if (tid == 255) wsum[0] = add + x;  // the round's inclusive total
        __syncthreads();
        carry = wsum[0];
        __syncthreads();
    }
    const int total = carry;
    if (tid == 0) {
        pre[S] = total;
        used_sh = 0;
    }
    __syncthreads();
    // keys >= thr are dropped: LCP below F, or (later) worse than the k-th held
    uint64_t thr = (uint64_t)(256 - F) << 32;
    int used = 0;
    auto sort_keep = [&]() {  // sorts keys[0, used) and keeps the best k
        int P = 1;
        while (P < used) P <<= 1;
        for (int t = used + tid; t < P; t += blockDim.x) keys[t] = kKeyInf;
        __syncthreads();
        for (int size = 2; size <= P; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int t = tid; t < P; t += blockDim.x) {
                    const int u = t ^ stride;
                    if (u > t) {
                        const uint64_t x = keys[t], y = keys[u];
                        const bool up = (t & size) == 0;
                        if ((x > y) == up) {
                            keys[t] = y;
                            keys[u] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
        if (used > k) used = k;
        if (used == k) thr = min(thr, keys[k - 1]);
        if (tid == 0) used_sh = used;
        __syncthreads();
    };
    constexpr int kRound = 1024;  // keys read per round, at most 4 a thread
    bool tight = false;           // thr already cut at a k-th key
    for (int base = 0; base < total;) {
        if (used + kRound > kMergeCap || (!tight && used >= k)) {  // block-uniform
            sort_keep();
            tight = used == k;
        }
        const int per = tight ? kRound / 256 : 1;  // one key a thread until the cut-off is set
#pragma unroll 4
        for (int e = 0; e < per; ++e) {
            const int g = base + e * 256 + tid;
            if (g < total) {
                int l = 0, h = S;  // the list holding key g: pre[l] <= g < pre[l + 1]
                while (h - l > 1) {
                    const int mid = (l + h) >> 1;
                    if (pre[mid] <= g) l = mid;
                    else h = mid;
                }
                const uint64_t v = lists[((int64_t)l * Q + qs) * cap + (g - pre[l])];
                if (v < thr) keys[atomicAdd(&used_sh, 1)] = v;
            }
        }
        base += per * 256;
        __syncthreads();
        used = used_sh;
    }
    sort_keep();
    for (int j = tid; j < k; j += blockDim.x) {
        const uint64_t v = j < used ? keys[j] : kKeyInf;
        out_ids[qi * k + j] = v == kKeyInf ? -1 : (int32_t)(uint32_t)v;
        out_lcp[qi * k + j] = v == kKeyInf ? 0 : (uint8_t)(255 - (int)(v >> 32));
    }
}

// ---- the batch order for the large-batch scan: queries by their first word ----

// keys[i] = packed word 0 of query i, vals[i] = i.
__global__ void k_query_keys(const uint8_t* __restrict__ queries, RowFmt qf, int64_t Q,
                             uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Q) return;
    keys[i] = pack_word(row_of(queries, i, qf), 0, qf);
    vals[i] = (uint32_t)i;
}

// One CTA: order[] = the query indices sorted by (word 0, index), Q <= kQuerySortCta.
__global__ void __launch_bounds__(1024) k_query_sort_cta(const uint8_t* __restrict__ queries, RowFmt qf, int Q,
                                                          int32_t* __restrict__ order) {
    extern __shared__ uint64_t qk[];  // [P] keys, then [P] indices
    int P = 1;
    while (P < Q) P <<= 1;
    uint32_t* qv = reinterpret_cast<uint32_t*>(qk + P);
    for (int t = threadIdx.x; t < P; t += blockDim.x) {
        qk[t] = t < Q ? pack_word(row_of(queries, t, qf), 0, qf) : ~0ull;
        qv[t] = (uint32_t)t;
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < P; t += blockDim.x) {
                const int u = t ^ stride;
                if (u > t) {
                    const uint64_t x = qk[t], y = qk[u];
                    const uint32_t vx = qv[t], vy = qv[u];
                    const bool gt = x > y || (x == y && vx > vy);
                    if (gt == ((t & size) == 0)) {
                        qk[t] = y;
                        qk[u] = x;
                        qv[t] = vy;
                        qv[u] = vx;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < Q; t += blockDim.x) order[t] = (int32_t)qv[t];
}

__global__ void k_u32_to_i32(const uint32_t* __restrict__ in, int64_t n, int32_t* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int32_t)in[i];
}

}  // namespace lcpk

namespace lcph {
using namespace lcpk;

// Larger batches: per-thread logs over N-slices, the batch ordered by the
// queries' first words (so that a warp's 32 queries are neighbours and its
// screen is narrow), each query's level floor taken first from a sample of
// the rows (the first kFloorSample: where k of them reach LCP d, no row
// below d can be in the answer), then the k-best merge.
constexpr int64_t kFloorSample = 65536;

// Resident k_scan_partial CTAs per multiprocessor (occupancy query, cached).
static int scan_ctas_per_sm() {
    static int cached = 0;
    if (!cached) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_scan_partial, kScanPartialThreads, 0) != cudaSuccess ||
            n < 1) {
            cudaGetLastError();
            n = 4;
        }
        cached = n;
    }
    return cached;
}

static int scan_logs(const void* d_tokens, int64_t N, const RowFmt& f, const void* d_queries, const RowFmt& qf,
                     int64_t Q, int k, int32_t* d_out_ids, uint8_t* d_out_lcp, cudaStream_t s) {
    const int threads = kScanPartialThreads;
    const int64_t qtiles = (Q + threads - 1) / threads;
    // CTAs of one full wave: slices per query tile rounded down to it (a
    // second, nearly empty wave costs more than a few idle slots)
    const int64_t target = (int64_t)sm_count() * scan_ctas_per_sm();
    auto slices = [&](int64_t rows, int64_t min_rows, int64_t max_s, int64_t* slice) {
        int64_t S = target / qtiles;
        const int64_t by_rows = (rows + min_rows - 1) / min_rows;
        if (S > by_rows) S = by_rows;
        if (S > max_s) S = max_s;
        if (S < 1) S = 1;
        *slice = ((rows + S - 1) / S + kScanSliceAlign - 1) / kScanSliceAlign * kScanSliceAlign;
        return (rows + *slice - 1) / *slice;
    };
    int64_t slice = 0;
    const int64_t S = slices(N, 1024, kMergeMaxLists, &slice);
    // the floor pass only pays when the sample is a small part of the rows
    const int64_t Ns = N >= 4 * kFloorSample ? kFloorSample : 0;
    int64_t slice_pre = 0;
    const int64_t S_pre = Ns ? slices(Ns, 4096, S, &slice_pre) : 0;
    const int cap = k + kLogSlack;  // log entries per (slice, query)
    const bool small_sort = Q <= kQuerySortCta;
    uint64_t *lists = nullptr, *qk0 = nullptr, *qk1 = nullptr;
    uint32_t *plane_hi = nullptr, *plane_lo = nullptr;
    int32_t *order = nullptr, *floor = nullptr, *counts = nullptr;
    uint32_t *qv0 = nullptr, *qv1 = nullptr;
    Carver cv;
    cv.add(&plane_hi, (size_t)N);
    cv.add(&plane_lo, (size_t)N);
    cv.add(&order, (size_t)Q);
    cv.add(&floor, (size_t)Q);
    cv.add(&counts, (size_t)S * Q);
    cv.add(&lists, (size_t)S * Q * cap);
    if (!small_sort) {
        cv.add(&qk0, (size_t)Q);
        cv.add(&qk1, (size_t)Q);
        cv.add(&qv0, (size_t)Q);
        cv.add(&qv1, (size_t)Q);
    }
    void* base = nullptr;
    LCP_CUDA_TRY(cv.alloc(&base, s));
    SortWork w;
    int rc = LCP_OK;
    if (!small_sort) rc = sort_work_alloc(w, (uint32_t)Q, lib_status_word(), s);
    cudaError_t e = cudaSuccess;
    if (rc == LCP_OK) {
        LCP_TIMED_LAUNCH(k_pack_plane0, (unsigned)((N + 255) / 256), 256, 0, s,
                         reinterpret_cast<const uint8_t*>(d_tokens), f, N, plane_hi, plane_lo);
        // the batch order
        if (small_sort) {
            int P = 1;
            while (P < Q) P <<= 1;
            const int smem = P * (int)(sizeof(uint64_t) + sizeof(uint32_t));
            e = cudaFuncSetAttribute(k_query_sort_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e == cudaSuccess)
                LCP_TIMED_LAUNCH(k_query_sort_cta, 1, 1024, smem, s, reinterpret_cast<const uint8_t*>(d_queries), qf,
                                 (int)Q, order);
        } else {
            LCP_TIMED_LAUNCH(k_query_keys, (unsigned)((Q + 255) / 256), 256, 0, s,
                             reinterpret_cast<const uint8_t*>(d_queries), qf, Q, qk0, qv0);
            uint64_t* ok = nullptr;
            uint32_t* ov = nullptr;
            rc = radix_sort_pairs_u64(qk0, qv0, qk1, qv1, (uint32_t)Q, 64, w, s, &ok, &ov);
            if (rc == LCP_OK) LCP_TIMED_LAUNCH(k_u32_to_i32, (unsigned)((Q + 255) / 256), 256, 0, s, ov, Q, order);
        }
    }
    if (rc == LCP_OK && e == cudaSuccess) e = cudaMemsetAsync(floor, 0, sizeof(int32_t) * (size_t)Q, s);
    ScanArgs a;
    a.tokens = reinterpret_cast<const uint8_t*>(d_tokens);
    a.plane_hi = plane_hi;
    a.plane_lo = plane_lo;
    a.f = f;
    a.queries = reinterpret_cast<const uint8_t*>(d_queries);
    a.qf = qf;
    a.Q = Q;
    a.order = order;
    a.k = k;
    a.cap = cap;
    a.lists = lists;
    a.status = lib_status_word();
    a.floor = floor;
    if (rc == LCP_OK && e == cudaSuccess && Ns) {  // the floors, from the sample
        a.N = Ns;
        a.slice = slice_pre;
        a.counts = nullptr;
        LCP_TIMED_LAUNCH(k_scan_partial, dim3((unsigned)qtiles, (unsigned)S_pre), threads, 0, s, a);
    }
    if (rc == LCP_OK && e == cudaSuccess) {
        a.N = N;
        a.slice = slice;
        a.counts = counts;
        LCP_TIMED_LAUNCH(k_scan_partial, dim3((unsigned)qtiles, (unsigned)S), threads, 0, s, a);
        e = cudaFuncSetAttribute(k_scan_merge, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(uint64_t) * kMergeCap));
        if (e == cudaSuccess)
            LCP_TIMED_LAUNCH(k_scan_merge, (unsigned)Q, 256, sizeof(uint64_t) * kMergeCap, s, lists, counts, cap, Q,
                             (int)S, k, order, d_out_ids, d_out_lcp);
    }
    if (rc == LCP_OK && e != cudaSuccess) rc = cuda_status(e);
    if (!small_sort && w.arena) sort_work_free(w, s);
    cudaFreeAsync(base, s);
    return rc;
}

int scan_topk_device(const void* d_tokens, int64_t N, int tb, int L, const void* d_queries,
                     int64_t Q, int k, int32_t* d_out_ids, uint8_t* d_out_lcp, cudaStream_t s) {
    if (Q <= 0) return LCP_OK;
    if (N <= 0) {
        LCP_CUDA_TRY(cudaMemsetAsync(d_out_ids, 0xFF, sizeof(int32_t) * (size_t)Q * k, s));
        LCP_CUDA_TRY(cudaMemsetAsync(d_out_lcp, 0, (size_t)Q * k, s));
        return LCP_OK;
    }
    RowFmt f = make_fmt(tb, L, d_tokens);
    RowFmt qf = make_fmt(tb, L, d_queries);
    if (Q <= kSelMaxQ) return scan_select(d_tokens, N, f, d_queries, qf, Q, k, d_out_ids, d_out_lcp, s);
    return scan_logs(d_tokens, N, f, d_queries, qf, Q, k, d_out_ids, d_out_lcp, s);
}

}  // namespace lcph
