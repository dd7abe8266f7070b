// Full scan top-k of small and middle batches by threshold selection: one
// read of the rows' first 16 bytes, no index (the paper's "full scan", Sec. 7
// Table 6, computing Definition "Top-k LCP Retrieval", Sec. 2.1).
//
// For a query, d* is the largest d with at least k rows of LCP >= d (0 when
// there is none).  Every row of LCP > d* is in the answer (fewer than k of
// them) and the remaining kp = min(k - nA, #rows of LCP d*) slots go to the
// rows of LCP exactly d* in ascending id: ties broken by index.
//
//   k_sel_count  the rows pass through shared memory in tiles of 256, each
//                row's first 16 bytes brought by a 2D bulk tensor copy (the
//                TMA unit; a 2-tile ring per warp, 64-byte L2 promotion), so
//                that the rows are read once for the whole batch.  A lane
//                per query counts, per tile (a "granule"), the rows of LCP
//                >= 1, 2, 3, 4 -- word 0 decides these -- and computes the
//                exact LCP of the few rows whose first tokens match: their
//                keys go to two per-query lists, rows of LCP >= 2 (uint16
//                tokens) and rows of LCP >= 4, each capped; rows of LCP > 4
//                also to a per-query level histogram.  From 160 queries a
//                warp sorts each full tile by word 0 first, and a query's
//                counts and matching rows are key ranges (binary searches)
//                instead of a pass over the tile.  It also writes word 0 of
//                every row (the plane) for the walks.
//   k_sel_answer a CTA per query (1,024, 512 or 256 threads as the batch
//                grows): the level totals, d*, nA and kp.  When
//                every row of LCP >= d* is listed (d* >= 4, or d* >= 2 with
//                the LCP >= 2 list complete), the list's k smallest keys are
//                written (an 8-bit radix select for long lists, then a sort).
//                Otherwise the answer rows not listed are located by
//                granule -- granules holding such rows of LCP > d*, and the
//                granules holding the first kp rows of LCP d* (a scan of the
//                per-granule tie counts) -- and the CTA's warps walk them,
//                reading the granule's words 0 in id order: unlisted rows of
//                LCP > d* join A, rows of LCP d* take their rank among the
//                ties; A (with the listed rows) is sorted and written.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "scan.cuh"

namespace lcpk {

constexpr int kSelRows = 256;    // rows per tile = per granule (one tensor-copy box)
constexpr int kSelList = 4096;    // keys of rows of LCP >= kSelDeep kept per query
constexpr int kSelDeep = 4;       // levels 1..kSelDeep are counted per granule
constexpr uint64_t kSelKeyInf = ~0ull;

struct SelArgs {
    const uint8_t* tokens;  // [N, L] raw rows
    RowFmt f;
    int64_t N;
    const uint8_t* queries;  // [Q, L] raw queries
    RowFmt qf;
    int Q, k;
    int64_t ngran;      // ceil(N / kSelRows)
    uint64_t* cnt;      // [Q][ngran]: 16-bit counts of rows with LCP >= 1, 2, 3, 4 (bits 0, 16, 32, 48)
    uint32_t* hist;     // [Q][L + 1]: rows of LCP exactly l, for l > kSelDeep (zeroed)
    uint64_t* list2;    // [Q][kSelList]: keys (255 - LCP) << 32 | id of rows with LCP >= 2 (uint16 tokens)
    uint64_t* list4;    // [Q][kSelList]: the same for rows with LCP >= kSelDeep
    uint32_t* n2;       // [Q]: keys appended to list2; > kSelList once a row did not fit (zeroed)
    uint32_t* n4;       // [Q]: the same for list4
    uint64_t* plane;    // [N]: packed word 0 of every row, for the walks
    int32_t* out_ids;   // [Q][k]
    uint8_t* out_lcp;   // [Q][k]
    int* status;
    int sorted;         // full tiles are sorted by word 0 and searched
    int stages;         // ring stages a warp (the CTA's warps: blockDim.x / 32)
};

__device__ __forceinline__ uint64_t sel_key(int l, int64_t id) {
    return ((uint64_t)(255 - l) << 32) | (uint64_t)(uint32_t)id;
}

// Exact LCP of a row with the query beyond word 1 (words 0 and 1 equal);
// qrow is the raw query.
__device__ int sel_lcp_deep(const uint8_t* row, const uint8_t* qrow, const RowFmt& f, const RowFmt& qf) {
    for (int w = 2; w < f.W; ++w) {
        const uint64_t y = pack_word(row, w, f) ^ pack_word(qrow, w, qf);
        if (y) return lcp_at(w, y, f);
    }
    return f.L;
}

// One 2D bulk tensor copy: the first 16 bytes of kSelRows rows starting at
// row y, completion counted on bar.
__device__ __forceinline__ void sel_tile_copy(const CUtensorMap* tm, void* dst, int y, uint64_t* bar) {
    mbar_arrive_expect_tx(bar, kSelRows * 16);
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(tm), "r"(0), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Each warp runs its own pipeline over tiles gw, gw + W, ... (gw its index
// in the grid, W the warps of the grid): a ring of tile
// buffers filled by tensor copies that its lane 0 issues, each tile
// converted in place (most significant token first) by the warp, then
// scanned by every chunk of 32 queries (a lane each, the tile's words read
// as broadcasts) -- no block-wide barrier after the start.  Rows whose first
// 32 bits match a query's get their exact LCP at once (word 1 is in the
// tile); those to be listed wait in a per-warp queue whose appends (global
// atomics) the warp issues together, 32 a round, once the queue might not
// hold another step's rows and at the end of the tile.  Dynamic shared memory: the
// warps' rings, their queues, their tile's upper halves and sorted rows,
// then the batch's words 0 and 1 (Q x 16 bytes) and two list-full flags per
// query.
// 12 warps a CTA with one ring stage each: 24 warps a multiprocessor (two
// CTAs fit the shared memory) with 24 tiles in flight, against 16 warps with
// two stages each (1 query 0.088 -> 0.086 ms, 32: 0.095 -> 0.092, 1,024
// sorted: 0.477 -> 0.439).
constexpr int kSelCountWarps = 12;
constexpr int kSelWarpStages = 1;
constexpr int kSelMaxWarps = kSelCountWarps;
constexpr int kSelMaxStages = kSelWarpStages;
constexpr int kSelQueue = 512;  // queued rows per warp
constexpr int kSelStep = 256;  // most rows one 8-row step of 32 queries can queue
// Batches from this size up search sorted tiles: sorting a tile by its
// 64-bit word 0 costs about as much as comparing four or five 32-query
// chunks with its rows, and every chunk then takes a few binary searches
// instead of a pass over the rows (measured on 2M rows of 64 uint16 tokens:
// 160 queries 0.179 ms compared, 0.174 sorted; 192 queries 0.203 / 0.186).
constexpr int kSelSortedMinQ = 160;

// Per warp: its ring, its queue, a tile's upper halves of word 0 and (sorted
// tiles) its rows in key order; then the batch's words 0 and 1 and two
// list-full flags per query.
__host__ __device__ constexpr size_t sel_warp_smem(int stages) {
    return (size_t)stages * kSelRows * 16 + (size_t)kSelQueue * sizeof(uint32_t) + (size_t)kSelRows * sizeof(uint32_t) +
           (size_t)kSelRows;
}
__host__ __device__ constexpr size_t sel_count_smem(int Q, int warps, int stages) {
    return (size_t)warps * sel_warp_smem(stages) + (size_t)Q * (2 * sizeof(uint64_t) + 2);
}

// One in-lane stage (distance J < 8) of the bitonic network below.
template <int J>
__device__ __forceinline__ void sort256_in_lane(uint64_t (&k)[8], uint32_t (&v)[8], unsigned lane, int size) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if ((i & J) == 0) {
            const int i2 = i | J;
            const bool up = ((lane * 8 + (unsigned)i) & (unsigned)size) == 0;
            if ((k[i] > k[i2]) == up) {
                const uint64_t tk = k[i];
                const uint32_t tv = v[i];
                k[i] = k[i2];
                v[i] = v[i2];
                k[i2] = tk;
                v[i2] = tv;
            }
        }
    }
}

// Ascending bitonic sort of 256 keys held 8 a lane (element 8 * lane + i) by
// one warp, each key carrying a value; equal keys end in either order.  The
// stage loops stay rolled: the kernel's code then fits the instruction cache.
__device__ __forceinline__ void warp_sort256(uint64_t (&k)[8], uint32_t (&v)[8]) {
    const unsigned lane = lane_id();
#pragma unroll 1
    for (int size = 2; size <= 256; size <<= 1) {
#pragma unroll 1
        for (int j = size >> 1; j >= 8; j >>= 1) {  // the pair spans two lanes
            const int lj = j >> 3;
            const bool lower = (lane & (unsigned)lj) == 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const bool up = ((lane * 8 + (unsigned)i) & (unsigned)size) == 0;
                const uint64_t ok = __shfl_xor_sync(0xffffffffu, k[i], lj);
                const uint32_t ov = __shfl_xor_sync(0xffffffffu, v[i], lj);
                const bool take = lower == up ? ok < k[i] : ok > k[i];
                if (take) {
                    k[i] = ok;
                    v[i] = ov;
                }
            }
        }
        if (size >= 8) sort256_in_lane<4>(k, v, lane, size);
        if (size >= 4) sort256_in_lane<2>(k, v, lane, size);
        sort256_in_lane<1>(k, v, lane, size);
    }
}

// Keys of a sorted 256-entry array below x (lower bound), or at most x.
__device__ __forceinline__ int sorted_below(const uint32_t* s, uint32_t x) {
    int pos = 0;
#pragma unroll
    for (int step = 128; step >= 1; step >>= 1)
        if (s[pos + step - 1] < x) pos += step;
    return pos + (s[pos] < x ? 1 : 0);  // only pos == 255 can still move
}
__device__ __forceinline__ int sorted_at_most(const uint32_t* s, uint32_t x) {
    int pos = 0;
#pragma unroll
    for (int step = 128; step >= 1; step >>= 1)
        if (s[pos + step - 1] <= x) pos += step;
    return pos + (s[pos] <= x ? 1 : 0);
}
// The same inside [b, e) of a sorted tile whose low key halves sit in the
// word-0 slots of the tile buffer (entry i at lw[4 * i]).
__device__ __forceinline__ int range_below(const uint32_t* lw, int b, int e, uint32_t x) {
    while (b < e) {
        const int m = (b + e) >> 1;
        if (lw[4 * m] < x) b = m + 1;
        else e = m;
    }
    return b;
}
__device__ __forceinline__ int range_at_most(const uint32_t* lw, int b, int e, uint32_t x) {
    while (b < e) {
        const int m = (b + e) >> 1;
        if (lw[4 * m] <= x) b = m + 1;
        else e = m;
    }
    return b;
}

template <int TB>
__global__ void __launch_bounds__(kSelMaxWarps * 32, 2) k_sel_count(const __grid_constant__ CUtensorMap tm,
                                                                   const SelArgs a, int use_tma) {
    extern __shared__ __align__(128) uint64_t dyn[];
    __shared__ __align__(8) uint64_t bar[kSelMaxWarps][kSelMaxStages];
    __shared__ uint32_t qn[kSelMaxWarps];
    const int warp = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    const int nwarps = (int)(blockDim.x >> 5);
    const int stages = a.stages;
    char* const base = reinterpret_cast<char*>(dyn);
    const size_t ring_b = (size_t)nwarps * stages * kSelRows * 16;
    const size_t queue_b = (size_t)nwarps * kSelQueue * sizeof(uint32_t);
    const size_t hi_b = (size_t)nwarps * kSelRows * sizeof(uint32_t);
    const size_t row_b = (size_t)nwarps * kSelRows;
    uint64_t (*ring)[kSelRows][2] = reinterpret_cast<uint64_t (*)[kSelRows][2]>(dyn) + warp * stages;
    uint32_t* queue = reinterpret_cast<uint32_t*>(base + ring_b) + warp * kSelQueue;
    // the current tile's upper halves of word 0, contiguous: four rows a 16-byte load
    uint32_t* hiw = reinterpret_cast<uint32_t*>(base + ring_b + queue_b) + warp * kSelRows;
    // a sorted tile's rows in the order of their sorted keys (kept in hiw)
    uint8_t* srow = reinterpret_cast<uint8_t*>(base + ring_b + queue_b + hi_b) + warp * kSelRows;
    uint64_t* qword0 = reinterpret_cast<uint64_t*>(base + ring_b + queue_b + hi_b + row_b);  // [Q] word 0
    uint64_t* qword1 = qword0 + a.Q;                                                          // [Q] and word 1
    uint8_t* full = reinterpret_cast<uint8_t*>(qword1 + a.Q);  // [Q][2]: list2 / list4 seen full
    uint64_t* wb = bar[warp];
    const RowFmt& f = a.f;
    const int64_t ntiles = a.ngran;
    const int64_t gw = (int64_t)blockIdx.x * nwarps + warp;
    const int64_t nw = (int64_t)gridDim.x * nwarps;
    const int nch = (a.Q + 31) / 32;
    const int L = f.L;
    // levels above L never occur: their thresholds are out of reach
    const int th2 = L >= 2 ? 2 : 99, th3 = L >= 3 ? 3 : 99, th4 = L >= 4 ? 4 : 99;
    for (int i = threadIdx.x; i < a.Q; i += blockDim.x) {
        const uint8_t* qrow = row_of(a.queries, i, a.qf);
        qword0[i] = pack_word(qrow, 0, a.qf);
        qword1[i] = f.W > 1 ? pack_word(qrow, 1, a.qf) : 0ull;
        full[2 * i] = 0;
        full[2 * i + 1] = 0;
    }
    if (lane == 0) {
        qn[warp] = 0;
        if (use_tma) {
            for (int s = 0; s < stages; ++s) mbar_init(&wb[s], 1);
            fence_proxy_async_smem();
        }
    }
    __syncthreads();
    if (use_tma && lane == 0)
        for (int s = 0; s < stages; ++s) {
            const int64_t t = gw + (int64_t)s * nw;
            if (t < ntiles) sel_tile_copy(&tm, ring[s], (int)(t * kSelRows), &wb[s]);
        }
    // the warp's queued rows (query, row in tile, LCP) into the capped
    // per-query lists: one atomic per (list, query) among a round's 32
    // entries (popular queries put many rows into one list); a CTA that met
    // a list's cap appends no more to it (its counter then exceeds the cap)
    const unsigned ltm = lanemask_lt();
    auto append = [&](uint64_t* list, uint32_t* n, int q, int which, uint64_t key, bool want) {
        want = want && !full[2 * q + which];
        const unsigned peers = __match_any_sync(0xffffffffu, want ? (uint32_t)q : 0xFFFFFFFFu);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (want && (int)lane == leader) base = atomicAdd(n + q, (uint32_t)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (!want) return;
        const uint32_t j = base + (uint32_t)__popc(peers & ltm);
        if (j < (uint32_t)kSelList) list[(size_t)q * kSelList + j] = key;
        else full[2 * q + which] = 1;
    };
    auto flush = [&](int64_t r0) {
        __syncwarp();
        const uint32_t n = qn[warp];
        for (uint32_t i0 = 0; i0 < n; i0 += 32) {
            const uint32_t i = i0 + lane;
            const bool in = i < n;
            const uint32_t e = in ? queue[i] : 0u;
            const int q = (int)(e >> 16), r = (int)((e >> 8) & 255u), l = (int)(e & 255u);
            const uint64_t key = sel_key(l, r0 + r);
            append(a.list2, a.n2, q, 0, key, in && TB == 2 && l >= 2);
            append(a.list4, a.n4, q, 1, key, in && l >= kSelDeep);
            if (in && l > kSelDeep) atomicAdd(a.hist + (size_t)q * (L + 1) + l, 1u);
        }
        __syncwarp();
        if (lane == 0) qn[warp] = 0;
        __syncwarp();
    };
    int it = 0;
    bool bad = false;
    for (int64_t t = gw; t < ntiles; t += nw, ++it) {
        const int s = it % stages;
        const int64_t r0 = t * kSelRows;
        const int nrows = a.N - r0 < kSelRows ? (int)(a.N - r0) : kSelRows;
        uint64_t (*buf)[2] = ring[s];
        if (use_tma) {
            bool ok = true;
            if (lane == 0) ok = mbar_wait(&wb[s], (uint32_t)((it / stages) & 1), kSpinLimit);
            if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) {
                bad = true;
                break;
            }
            for (int r = (int)lane; r < nrows; r += 32) {
                const uint64_t x0 = msb_first(buf[r][0], TB);
                buf[r][0] = x0;
                hiw[r] = (uint32_t)(x0 >> 32);
                buf[r][1] = msb_first(buf[r][1], TB);
                a.plane[r0 + r] = x0;
            }
        } else {
            for (int r = (int)lane; r < nrows; r += 32) {
                const uint8_t* row = row_of(a.tokens, r0 + r, f);
                const uint64_t x0 = pack_word(row, 0, f);
                buf[r][0] = x0;
                hiw[r] = (uint32_t)(x0 >> 32);
                buf[r][1] = f.W > 1 ? pack_word(row, 1, f) : 0ull;
                a.plane[r0 + r] = x0;
            }
        }
        __syncwarp();
        // a full tile of a larger batch: sorted by word 0 (its rows beside
        // it), so that a query's level counts are the widths of key ranges
        // and the rows it has to look at one range.  The sorted upper halves
        // go to hiw, the lower halves to the word-0 slots of the tile buffer
        // (entry i at buf[i][0]); word 1 stays in place, found through srow.
        const bool srt = a.sorted && nrows == kSelRows;
        if (srt) {
            uint64_t kk[8];
            uint32_t vv[8];
            const uint4* h4 = reinterpret_cast<const uint4*>(hiw) + lane * 2;
            const uint4 u = h4[0], v = h4[1];
            const uint32_t hk[8] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                vv[i] = lane * 8 + (unsigned)i;
                kk[i] = ((uint64_t)hk[i] << 32) | (uint32_t)buf[lane * 8 + i][0];
            }
            warp_sort256(kk, vv);
            __syncwarp();  // every lane has read its keys
            uint4* o4 = reinterpret_cast<uint4*>(hiw) + lane * 2;
            o4[0] = make_uint4((uint32_t)(kk[0] >> 32), (uint32_t)(kk[1] >> 32), (uint32_t)(kk[2] >> 32),
                               (uint32_t)(kk[3] >> 32));
            o4[1] = make_uint4((uint32_t)(kk[4] >> 32), (uint32_t)(kk[5] >> 32), (uint32_t)(kk[6] >> 32),
                               (uint32_t)(kk[7] >> 32));
#pragma unroll
            for (int i = 0; i < 8; ++i) buf[lane * 8 + i][0] = (uint32_t)kk[i];
            reinterpret_cast<uint2*>(srow)[lane] = make_uint2(vv[0] | vv[1] << 8 | vv[2] << 16 | vv[3] << 24,
                                                              vv[4] | vv[5] << 8 | vv[6] << 16 | vv[7] << 24);
            __syncwarp();
        }
        for (int c = 0; c < nch; ++c) {
            const int q = c * 32 + (int)lane;
            const bool qa = q < a.Q;
            const uint64_t q0 = qa ? qword0[q] : 0ull;
            const uint32_t qh = qa ? (uint32_t)(q0 >> 32) : ~(uint32_t)buf[0][0];  // inactive lanes never match
            const uint32_t ql = (uint32_t)q0;
            uint32_t c1 = 0, c2 = 0, c3 = 0, c4 = 0;
            // a row whose first 32 bits (2 uint16 / 4 uint8 tokens) match the
            // query's: exact LCP, level counts, queued if it is to be listed
            // a row whose first 32 bits (2 uint16 / 4 uint8 tokens) match the
            // query's: its exact LCP (lw = the lower half of its word 0), the
            // level counts when they are not taken from ranges, and queued
            // if it is to be listed
            auto deep = [&](int r, uint32_t lw, bool count) {
                if (!qa) return;
                int l;
                const uint32_t xl = lw ^ ql;
                if (xl) {
                    l = lcp_at(0, (uint64_t)xl, f);
                } else if (f.W == 1) {
                    l = L;
                } else {
                    const uint64_t x1 = buf[r][1] ^ qword1[q];
                    l = x1 ? lcp_at(1, x1, f)
                           : (f.W > 2 ? sel_lcp_deep(row_of(a.tokens, r0 + r, f), row_of(a.queries, q, a.qf), f, a.qf)
                                      : L);
                }
                if (TB == 2 && count) {
                    c2 += l >= th2;
                    c3 += l >= th3;
                    c4 += l >= th4;
                }
                // queued for a list this CTA has not seen full, or for the histogram
                const bool w2 = TB == 2 && l >= 2 && !full[2 * q];
                const bool w4 = l >= kSelDeep && !full[2 * q + 1];
                if (w2 || w4 || l > kSelDeep)
                    queue[atomicAdd(&qn[warp], 1u)] = ((uint32_t)q << 16) | ((uint32_t)r << 8) | (uint32_t)l;
            };
            if (srt) {
                // rows whose first d tokens equal q's: keys between q's key
                // with the bits past those tokens cleared and with them set
                auto width = [&](uint32_t low_bits) {
                    return (uint32_t)(sorted_at_most(hiw, qh | low_bits) - sorted_below(hiw, qh & ~low_bits));
                };
                const uint32_t* lws = reinterpret_cast<const uint32_t*>(buf);
                int lo = qa ? sorted_below(hiw, qh) : 0;  // [lo, hi): the first 32 bits match
                int hi = qa ? sorted_at_most(hiw, qh) : 0;
                if (qa) {
                    if (TB == 2) {
                        c1 = width(0xFFFFu);
                        if (hi > lo) {
                            // tokens 2 and 3 inside the range, ordered by the lower halves
                            const int lo3 = range_below(lws, lo, hi, ql & 0xFFFF0000u);
                            const int hi3 = range_at_most(lws, lo3, hi, ql | 0xFFFFu);
                            const int lo4 = range_below(lws, lo3, hi3, ql);
                            const int hi4 = range_at_most(lws, lo4, hi3, ql);
                            c2 = L >= 2 ? (uint32_t)(hi - lo) : 0u;
                            c3 = L >= 3 ? (uint32_t)(hi3 - lo3) : 0u;
                            c4 = L >= 4 ? (uint32_t)(hi4 - lo4) : 0u;
                            // rows of LCP 2 and 3 matter only to a list not yet full
                            if (full[2 * q]) lo = lo4, hi = hi4;
                        }
                    } else {
                        c1 = width(0xFFFFFFu);
                        c2 = L >= 2 ? width(0xFFFFu) : 0u;
                        c3 = L >= 3 ? width(0xFFu) : 0u;
                        c4 = L >= 4 ? (uint32_t)(hi - lo) : 0u;
                    }
                }
                // the rows to look at: 8 a lane a round
                for (; __any_sync(0xffffffffu, lo < hi); lo += 8) {
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (lo + j < hi) deep((int)srow[lo + j], lws[4 * (lo + j)], false);
                    __syncwarp();
                    if (qn[warp] > (uint32_t)(kSelQueue - kSelStep)) flush(r0);
                }
                if (qa)
                    a.cnt[(size_t)q * a.ngran + t] =
                        ((uint64_t)(c3 | (c4 << 16)) << 32) | (uint64_t)(c1 | (c2 << 16));
                continue;
            }
            int r = 0;
            const uint4* h4 = reinterpret_cast<const uint4*>(hiw);
            for (; r + 8 <= nrows; r += 8) {
                const uint4 u = h4[r >> 2], v = h4[(r >> 2) + 1];  // broadcasts
                const uint32_t x[8] = {u.x ^ qh, u.y ^ qh, u.z ^ qh, u.w ^ qh, v.x ^ qh, v.y ^ qh, v.z ^ qh, v.w ^ qh};
                uint32_t m = ~0u;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint32_t xh = x[j];
                    if (TB == 2) {
                        c1 += xh < (1u << 16) ? 1u : 0u;
                    } else {
                        const int l0 = __clz(xh) >> 3;
                        c1 += l0 >= 1 ? 1u : 0u;
                        c2 += l0 >= th2 ? 1u : 0u;
                        c3 += l0 >= th3 ? 1u : 0u;
                        c4 += l0 >= th4 ? 1u : 0u;
                    }
                    m = min(m, xh);
                }
                if (!qa) m = ~0u;
                if (__any_sync(0xffffffffu, m == 0)) {  // rare: at most kSelStep rows queued
                    if (m == 0)
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (x[j] == 0) deep(r + j, (uint32_t)buf[r + j][0], true);
                    __syncwarp();
                    if (qn[warp] > (uint32_t)(kSelQueue - kSelStep)) flush(r0);
                }
            }
            for (; r < nrows; ++r) {
                const uint32_t xh = hiw[r] ^ qh;
                if (TB == 2) {
                    c1 += xh < (1u << 16) ? 1u : 0u;
                } else {
                    const int l0 = __clz(xh) >> 3;
                    c1 += l0 >= 1 ? 1u : 0u;
                    c2 += l0 >= th2 ? 1u : 0u;
                    c3 += l0 >= th3 ? 1u : 0u;
                    c4 += l0 >= th4 ? 1u : 0u;
                }
                if (__any_sync(0xffffffffu, qa && xh == 0)) {
                    if (qa && xh == 0) deep(r, (uint32_t)buf[r][0], true);
                    __syncwarp();
                    if (qn[warp] > (uint32_t)(kSelQueue - kSelStep)) flush(r0);
                }
            }
            if (qa)
                a.cnt[(size_t)q * a.ngran + t] = ((uint64_t)(c3 | (c4 << 16)) << 32) | (uint64_t)(c1 | (c2 << 16));
        }
        __syncwarp();
        if (qn[warp] != 0) flush(r0);  // the queued rows name rows of this tile
        __syncwarp();  // every lane is done with the buffer
        if (use_tma && lane == 0) {
            const int64_t tn = t + (int64_t)stages * nw;
            // the warp's reads and in-place writes come before the copy's writes
            fence_proxy_async_smem();
            if (tn < ntiles) sel_tile_copy(&tm, ring[s], (int)(tn * kSelRows), &wb[s]);
        }
    }
    if (bad && lane == 0) {
        flag_status(a.status, DEV_TIMEOUT);
        // copies still in flight land before the CTA's shared memory is reused
        for (int j = 0; j < stages; ++j) {
            const int i = it + j;
            const int64_t t = gw + (int64_t)i * nw;
            if (t < ntiles) (void)mbar_wait(&wb[i % stages], (uint32_t)((i / stages) & 1), kSpinLimit);
        }
    }
}

__device__ __forceinline__ uint32_t cnt_level(uint64_t v, int d) {  // rows of LCP >= d, d = 1..4
    return (uint32_t)(v >> (16 * (d - 1))) & 0xFFFFu;
}

// Bitonic sort of P (a power of two) keys in shared memory by the threads of
// the block.
__device__ void sel_sort_block(uint64_t* keys, int P) {
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < P; t += blockDim.x) {
                const int u = t ^ stride;
                if (u > t) {
                    const uint64_t x = keys[t], y = keys[u];
                    if ((x > y) == ((t & size) == 0)) {
                        keys[t] = y;
                        keys[u] = x;
                    }
                }
            }
            __syncthreads();
        }
}

// Sorts keys[0, n) when they are unique: up to 256 of them by rank (thread
// t counts the keys below keys[t], all reading the same key at once, then
// writes its key to that slot: two barriers), more by the bitonic sort of
// the P >= n keys (padding included).
__device__ void sel_sort_keys(uint64_t* keys, int n, int P) {
    if (n > 256 || n > (int)blockDim.x) {
        sel_sort_block(keys, P);
        return;
    }
    const int t = threadIdx.x;
    uint64_t mine = 0;
    int rank = 0;
    if (t < n) {
        mine = keys[t];
        int j = 0;
        for (; j + 4 <= n; j += 4)
            rank += (keys[j] < mine ? 1 : 0) + (keys[j + 1] < mine ? 1 : 0) + (keys[j + 2] < mine ? 1 : 0) +
                    (keys[j + 3] < mine ? 1 : 0);
        for (; j < n; ++j) rank += keys[j] < mine ? 1 : 0;
    }
    __syncthreads();
    if (t < n) keys[rank] = mine;
    __syncthreads();
}

__device__ __forceinline__ void sel_out(const SelArgs& a, int q, int j, int32_t id, int l) {
    a.out_ids[(size_t)q * a.k + j] = id;
    a.out_lcp[(size_t)q * a.k + j] = (uint8_t)l;
}

// Writes keys[0, n) (sorted) then the ties tbuf[0, nt) at level dstar, then
// padding, by the threads of a block (nthr, tid) or of a warp.
__device__ void sel_write(const SelArgs& a, int q, const uint64_t* keys, int n, const int32_t* tie, int nt, int dstar,
                          int tid, int nthr) {
    for (int j = tid; j < a.k; j += nthr) {
        if (j < n) {
            const uint64_t v = keys[j];
            sel_out(a, q, j, (int32_t)(uint32_t)v, 255 - (int)(v >> 32));
        } else if (j < n + nt) {
            sel_out(a, q, j, __ldcg(tie + (j - n)), dstar);
        } else {
            sel_out(a, q, j, -1, 0);
        }
    }
}

constexpr int kSelSortDirect = 256;  // lists up to this long are sorted whole

// The r-th smallest (1-based) of n unique 40-bit keys in shared memory, by
// the threads of the block: five 8-bit digit histograms over the keys that
// share the digits chosen so far (warp-aggregated shared-memory counts).
__device__ uint64_t sel_select_block(const uint64_t* keys, int n, int r) {
    __shared__ uint32_t bins[256];
    __shared__ uint64_t pre_s;
    __shared__ int rank_s;
    uint64_t pre = 0, pmask = 0;
    int rank = r;
    for (int shift = 32; shift >= 0; shift -= 8) {
        for (int t = threadIdx.x; t < 256; t += blockDim.x) bins[t] = 0;
        __syncthreads();
        for (int t0 = 0; t0 < n; t0 += blockDim.x) {
            const int t = t0 + threadIdx.x;
            const bool in = t < n && (keys[t] & pmask) == pre;
            const uint32_t d = in ? (uint32_t)(keys[t] >> shift) & 255u : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (in && lane_id() == (unsigned)(__ffs(peers) - 1)) atomicAdd(&bins[d], (uint32_t)__popc(peers));
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            // the digit whose bin holds the rank-th key: 8 bins per lane
            uint32_t c[8], sum = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                c[j] = bins[threadIdx.x * 8 + j];
                sum += c[j];
            }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane_id() >= (unsigned)o) incl += y;
            }
            uint32_t run = incl - sum;
            if (run < (uint32_t)rank && (uint32_t)rank <= incl) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (run < (uint32_t)rank && (uint32_t)rank <= run + c[j]) {
                        pre_s = pre | ((uint64_t)(threadIdx.x * 8 + j) << shift);
                        rank_s = rank - (int)run;
                    }
                    run += c[j];
                }
            }
        }
        __syncthreads();
        pre = pre_s;
        rank = rank_s;
        pmask |= 255ull << shift;
        __syncthreads();
    }
    return pre;
}

constexpr int kPickCache = 8;  // granule counts a pick thread keeps in registers
// Threads of an answer CTA (a query).  At 64 registers a thread the register
// file holds 1,024 threads a multiprocessor: one CTA of 1,024, two of 512 or
// four of 256.  Narrower CTAs let other queries' work overlap one query's
// barrier waits once the batch passes a wave: 1,024 threads up to two
// queries a multiprocessor, 512 up to three, 256 above (1,024 queries:
// answer 0.155 -> 0.136 -> 0.110 ms; 297 queries are faster at 512 than at
// 256, 32 queries at 1,024 than at 512, 0.035 / 0.040 ms).
constexpr int kSelAnswerWide = 1024;
constexpr int kSelAnswerMid = 512;
constexpr int kSelAnswerNarrow = 256;

// Dynamic shared memory: kSelList keys (a list, or the walk's items and then
// A), then k keys of the walk's A rows and k tie ids.
__global__ void __launch_bounds__(kSelAnswerWide) k_sel_answer(const SelArgs a) {
    extern __shared__ __align__(16) uint64_t keys[];  // kSelList keys (list mode, scan mode's A)
    __shared__ uint32_t lev[LCP_MAX_L + 2];           // rows with LCP >= d
    __shared__ uint32_t hs[LCP_MAX_L + 2];            // rows with LCP == l (l > kSelDeep)
    __shared__ uint32_t wsum[32][4];
    __shared__ uint32_t sh[8];
    const int q = blockIdx.x;
    const int L = a.f.L, k = a.k;
    const int tid = threadIdx.x;
    const unsigned lane = lane_id();
    const int warp = tid >> 5, nwarps = blockDim.x >> 5;
    const uint64_t* cq = a.cnt + (size_t)q * a.ngran;
    // each thread's granules: a contiguous run, the first kPickCache of them
    // loaded once into registers (all loads issued together)
    const int64_t per = (a.ngran + blockDim.x - 1) / blockDim.x;
    const int64_t gb = (int64_t)tid * per;
    const int64_t ge = gb + per < a.ngran ? gb + per : a.ngran;
    uint64_t cv[kPickCache];
#pragma unroll
    for (int j = 0; j < kPickCache; ++j) cv[j] = gb + j < ge ? cq[gb + j] : 0ull;
    // fn(g, count word) over the thread's granules in order: the cached
    // ones by constant register index, the rest from memory
    auto each_granule = [&](auto&& fn) {
#pragma unroll
        for (int j = 0; j < kPickCache; ++j)
            if (gb + j < ge) fn(gb + j, cv[j]);
        for (int64_t g = gb + kPickCache; g < ge; ++g) fn(g, cq[g]);
    };
    for (int l = tid; l <= L; l += blockDim.x) hs[l] = l > kSelDeep ? a.hist[(size_t)q * (L + 1) + l] : 0u;
    // level totals 1..4 over the granules
    uint32_t s1 = 0, s2 = 0, s3 = 0, s4 = 0;
    each_granule([&](int64_t, uint64_t v) {
        s1 += cnt_level(v, 1);
        s2 += cnt_level(v, 2);
        s3 += cnt_level(v, 3);
        s4 += cnt_level(v, 4);
    });
    s1 = __reduce_add_sync(0xffffffffu, s1);
    s2 = __reduce_add_sync(0xffffffffu, s2);
    s3 = __reduce_add_sync(0xffffffffu, s3);
    s4 = __reduce_add_sync(0xffffffffu, s4);
    if (lane == 0) {
        wsum[warp][0] = s1;
        wsum[warp][1] = s2;
        wsum[warp][2] = s3;
        wsum[warp][3] = s4;
    }
    __syncthreads();
    if (tid < 4) {
        uint32_t v = 0;
        for (int w = 0; w < nwarps; ++w) v += wsum[w][tid];
        if (tid + 1 <= L) lev[tid + 1] = v;
    } else if (tid == 32 && L > kSelDeep) {
        // deeper levels: suffix sums of the histogram (one warp)
        uint32_t carry = 0;
        for (int d = L; d > kSelDeep; --d) {
            carry += hs[d];
            lev[d] = carry;
        }
    }
    __syncthreads();
    // the counts fall with d: d* is the number of d in 1..L reaching k
    const int dstar = __syncthreads_count(tid >= 1 && tid <= L && lev[tid] >= (uint32_t)k);
    const uint32_t nA = dstar < L ? lev[dstar + 1] : 0u;
    const uint32_t atd = dstar == 0 ? (uint32_t)a.N : lev[dstar];
    const uint32_t kp = min((uint32_t)k - nA, atd - nA);
    const uint32_t n2 = a.n2[q], n4 = a.n4[q];
    const bool have2 = a.f.tb == 2 && n2 <= (uint32_t)kSelList;  // every row of LCP >= 2 listed
    const bool have4 = n4 <= (uint32_t)kSelList;
    // sorts a list's nl keys (every row of LCP >= d* among them) and writes
    // its first nw
    auto from_list = [&](const uint64_t* list, int nl, int nw) {
        const uint64_t* lq = list + (size_t)q * kSelList;
        int n = nl;
        if (nl > kSelSortDirect && nw < nl) {
            // long list: the nw-th smallest key by an 8-bit radix select over
            // the key's 40 bits (keys are unique), then only the keys up to
            // it are kept and sorted
            for (int t = tid; t < nl; t += blockDim.x) keys[t] = lq[t];
            const uint64_t kth = sel_select_block(keys, nl, nw);
            if (tid == 0) sh[2] = 0;
            __syncthreads();
            uint64_t mine[kSelList / kSelAnswerNarrow];
            int nm = 0;
            for (int t = tid; t < nl; t += blockDim.x)
                if (keys[t] <= kth) mine[nm++] = keys[t];
            __syncthreads();
            for (int j = 0; j < nm; ++j) keys[atomicAdd(&sh[2], 1u)] = mine[j];
            n = nw;
        } else {
            for (int t = tid; t < nl; t += blockDim.x) keys[t] = lq[t];
        }
        int P = 1;
        while (P < n) P <<= 1;
        for (int t = n + tid; t < P; t += blockDim.x) keys[t] = kSelKeyInf;
        __syncthreads();
        sel_sort_keys(keys, n, P);  // keys carry unique ids
        sel_write(a, q, keys, nw, nullptr, 0, dstar, tid, blockDim.x);
    };
    if ((dstar >= kSelDeep && have4) || (dstar >= 2 && have2)) {
        // every row of LCP >= d* is listed (at least k of them): the k
        // smallest keys of the shorter such list
        if (dstar >= kSelDeep && have4) from_list(a.list4, (int)n4, k);
        else from_list(a.list2, (int)n2, k);
        return;
    }
    if (dstar >= kSelDeep) {
        // more rows share the query's first kSelDeep tokens than the list
        // holds (heavy duplication): one pass over all rows in id order,
        // exact LCPs, A into shared memory, the first kp ties ranked
        const uint8_t* qrow = row_of(a.queries, q, a.qf);
        __shared__ uint32_t na_s, nt_s;
        __shared__ int32_t ties[LCP_SCAN_MAX_K];
        if (tid == 0) {
            na_s = 0;
            nt_s = 0;
        }
        __syncthreads();
        for (int64_t b = 0; b < a.N; b += blockDim.x) {
            const int64_t i = b + tid;
            int l = -1;
            if (i < a.N) {
                const uint8_t* row = row_of(a.tokens, i, a.f);
                l = a.f.L;
                for (int w = 0; w < a.f.W; ++w) {
                    const uint64_t y = pack_word(row, w, a.f) ^ pack_word(qrow, w, a.qf);
                    if (y) {
                        l = lcp_at(w, y, a.f);
                        break;
                    }
                }
            }
            if (l > dstar) {  // fewer than k such rows in all
                const uint32_t j = atomicAdd(&na_s, 1u);
                if (j < (uint32_t)kSelList) keys[j] = sel_key(l, i);
            }
            const bool isT = l == dstar;
            const unsigned mt = __ballot_sync(0xffffffffu, isT);
            if (lane == 0) wsum[warp][0] = __popc(mt);
            __syncthreads();
            uint32_t before = nt_s;
            for (int w = 0; w < warp; ++w) before += wsum[w][0];
            const uint32_t rank = before + __popc(mt & lanemask_lt());
            if (isT && rank < kp) ties[rank] = (int32_t)i;
            __syncthreads();
            if (tid == 0) {
                uint32_t add = 0;
                for (int w = 0; w < nwarps; ++w) add += wsum[w][0];
                nt_s += add;
            }
            __syncthreads();
            if (na_s >= nA && nt_s >= kp) break;
        }
        int P = 1;
        while (P < (int)nA) P <<= 1;
        for (int t = (int)nA + tid; t < P; t += blockDim.x) keys[t] = kSelKeyInf;
        __syncthreads();
        sel_sort_keys(keys, (int)nA, P);
        for (int j = tid; j < k; j += blockDim.x) {
            if (j < (int)nA) {
                const uint64_t v = keys[j];
                sel_out(a, q, j, (int32_t)(uint32_t)v, 255 - (int)(v >> 32));
            } else if (j < (int)(nA + kp)) {
                sel_out(a, q, j, ties[j - nA], dstar);
            } else {
                sel_out(a, q, j, -1, 0);
            }
        }
        return;
    }
    // d* < kSelDeep and not all rows of LCP >= d* listed.  Rows of LCP >= lt
    // are all listed (fewer than k of them, all in A): lt = 2 when the LCP >=
    // 2 list is complete (always for d* <= 1 with uint16 tokens), else
    // kSelDeep.  The CTA's warps walk the granules holding the rest: rows of
    // LCP in (d*, lt), and the first kp rows of LCP d* (ties before each
    // granule by an exclusive scan over the threads' runs).
    const int lt = have2 ? 2 : kSelDeep;
    uint4* items = reinterpret_cast<uint4*>(keys);  // at most nA + kp <= 2k of them
    uint64_t* abuf = keys + kSelList;                // [k] unlisted rows of LCP > d*
    int32_t* tbuf = reinterpret_cast<int32_t*>(abuf + k);  // [k] the first kp ties
    auto tie_count = [&](int64_t g, uint64_t v) -> uint32_t {
        const uint32_t at = dstar == 0 ? (uint32_t)min((int64_t)kSelRows, a.N - g * kSelRows) : cnt_level(v, dstar);
        return at - cnt_level(v, dstar + 1);
    };
    auto a_count = [&](uint64_t v) -> uint32_t {
        return dstar + 1 < lt ? cnt_level(v, dstar + 1) - cnt_level(v, lt) : 0u;
    };
    uint32_t tsum = 0;
    each_granule([&](int64_t g, uint64_t c) { tsum += tie_count(g, c); });
    uint32_t v = tsum;  // inclusive scan over the block
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= (unsigned)o) v += y;
    }
    if (lane == 31) wsum[warp][0] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (int)lane < nwarps ? wsum[lane][0] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= (unsigned)o) w += y;
        }
        wsum[lane][1] = w;
    }
    __syncthreads();
    const uint32_t tbase = v - tsum + (warp > 0 ? wsum[warp - 1][1] : 0u);
    // items, in any order (each carries its ties-before count): slots from a
    // shared counter
    if (tid == 0) {
        sh[0] = 0;  // items of this query
        sh[3] = 0;  // walk's A slots taken
    }
    __syncthreads();
    {
        uint32_t run = tbase;
        each_granule([&](int64_t g, uint64_t c) {
            const uint32_t tc = tie_count(g, c), ac = a_count(c);
            if (ac > 0 || (tc > 0 && run < kp)) {
                const uint32_t slot = atomicAdd(&sh[0], 1u);
                if (slot < (uint32_t)(2 * k)) items[slot] = make_uint4((uint32_t)g, run, ac, 0u);
            }
            run += tc;
        });
    }
    __syncthreads();
    const uint32_t nq = sh[0];
    // the walk: a warp per item, the granule's words 0 in id order
    {
        const RowFmt& f = a.f;
        const uint64_t q0 = pack_word(row_of(a.queries, q, a.qf), 0, a.qf);
        const unsigned ltm = lanemask_lt();
        for (uint32_t i = warp; i < nq && i < (uint32_t)(2 * k); i += nwarps) {
            const uint4 itm = items[i];
            const int64_t r0 = (int64_t)itm.x * kSelRows;
            const int64_t r1 = r0 + kSelRows < a.N ? r0 + kSelRows : a.N;
            uint32_t seen = itm.y;  // ties before this row group
            const bool want_a = itm.z > 0;
            uint64_t w[kSelRows / 32];
#pragma unroll
            for (int j = 0; j < kSelRows / 32; ++j) {  // all loads issued first
                const int64_t r = r0 + j * 32 + lane;
                w[j] = r < r1 ? a.plane[r] : q0;
            }
#pragma unroll
            for (int j = 0; j < kSelRows / 32; ++j) {
                if (!want_a && seen >= kp) break;  // warp-uniform
                const int64_t r = r0 + j * 32 + lane;
                const uint64_t x = w[j] ^ q0;
                // LCP from word 0 (exact below kSelDeep; rows of LCP >= lt are listed)
                const int l = x ? lcp_at(0, x, f) : (f.tpw < f.L ? f.tpw : f.L);
                const bool in = r < r1;
                const bool isA = in && l > dstar && l < lt;
                const bool isT = in && l == dstar;
                const unsigned mA = __ballot_sync(0xffffffffu, isA);
                if (mA) {
                    uint32_t base = 0;
                    if (lane == 0) base = atomicAdd(&sh[3], (uint32_t)__popc(mA));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    const uint32_t slot = base + (uint32_t)__popc(mA & ltm);
                    if (isA) {
                        if (slot < (uint32_t)k) abuf[slot] = sel_key(l, r);
                        else flag_status(a.status, DEV_BAD);  // never for consistent counts
                    }
                }
                const unsigned mT = __ballot_sync(0xffffffffu, isT);
                if (isT) {
                    const uint32_t rank = seen + (uint32_t)__popc(mT & ltm);
                    if (rank < kp) tbuf[rank] = (int32_t)r;
                }
                seen += (uint32_t)__popc(mT);
            }
        }
    }
    __syncthreads();
    // A: the walk's rows and the listed ones (all of LCP >= lt > d*), sorted
    const int nw_a = min((int)sh[3], k);
    const int nl = min((int)(lt == 2 ? n2 : n4), k - nw_a);
    const int n = nw_a + nl;
    const uint64_t* lq = (lt == 2 ? a.list2 : a.list4) + (size_t)q * kSelList;
    int P = 1;
    while (P < n) P <<= 1;
    for (int t = tid; t < P; t += blockDim.x) keys[t] = t < nw_a ? abuf[t] : (t < n ? lq[t - nw_a] : kSelKeyInf);
    __syncthreads();
    sel_sort_keys(keys, n, P);  // the walk's rows are not listed: unique ids
    for (int j = tid; j < k; j += blockDim.x) {
        if (j < n) {
            const uint64_t x = keys[j];
            sel_out(a, q, j, (int32_t)(uint32_t)x, 255 - (int)(x >> 32));
        } else if (j < n + (int)kp) {
            sel_out(a, q, j, tbuf[j - n], dstar);
        } else {
            sel_out(a, q, j, -1, 0);
        }
    }
}

}  // namespace lcpk

namespace lcph {
using namespace lcpk;

// cuTensorMapEncodeTiled, through the runtime's driver entry point (no link
// against libcuda).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        cudaDriverEntryPointQueryResult qr;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) ==
                cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// The tensor map of the rows' first 16 bytes (box: 16 bytes x kSelRows rows),
// when the layout allows one: 16-byte aligned base, row pitch a multiple of
// 16 bytes and rows of at least 16 bytes.
static bool sel_tensor_map(const void* tokens, int64_t N, const RowFmt& f, CUtensorMap* tm) {
    if ((reinterpret_cast<uintptr_t>(tokens) & 15) || f.row_bytes % 16 || f.row_bytes < 16 || N >= (1ll << 31))
        return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)f.L, (cuuint64_t)N};
    cuuint64_t strides[1] = {(cuuint64_t)f.row_bytes};
    cuuint32_t box[2] = {(cuuint32_t)(16 / f.tb), (cuuint32_t)kSelRows};
    cuuint32_t es[2] = {1, 1};
    const CUresult r = enc(tm, f.tb == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                           const_cast<void*>(tokens), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_64B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

static size_t sel_answer_smem(int k) { return kSelList * sizeof(uint64_t) + (size_t)k * (sizeof(uint64_t) + 4); }

// Per-device launch set-up, done once: the answer kernel's shared-memory limit (k up
// to LCP_SCAN_MAX_K) and the count kernel's resident CTAs per multiprocessor
// at the largest batch.
struct SelSetup {
    int count_ctas[2] = {0, 0};  // uint8, uint16 tokens
    bool ok = false;
};

static const SelSetup* sel_setup() {
    static SelSetup st[64];
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    SelSetup& x = st[dev];
    if (x.ok) return &x;
    const size_t count_smem = sel_count_smem((int)kSelMaxQ, kSelCountWarps, kSelWarpStages);
    if (cudaFuncSetAttribute(k_sel_answer, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sel_answer_smem(LCP_SCAN_MAX_K)) != cudaSuccess ||
        cudaFuncSetAttribute(k_sel_count<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)count_smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_sel_count<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)count_smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&x.count_ctas[0], k_sel_count<1>, kSelCountWarps * 32,
                                                      count_smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&x.count_ctas[1], k_sel_count<2>, kSelCountWarps * 32,
                                                      count_smem) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    for (int& c : x.count_ctas)
        if (c < 1) c = 1;
    x.ok = true;
    return &x;
}

int scan_select(const void* d_tokens, int64_t N, const RowFmt& f, const void* d_queries, const RowFmt& qf,
                int64_t Q, int k, int32_t* d_out_ids, uint8_t* d_out_lcp, cudaStream_t s) {
    const int L = f.L;
    SelArgs a;
    a.tokens = reinterpret_cast<const uint8_t*>(d_tokens);
    a.f = f;
    a.N = N;
    a.queries = reinterpret_cast<const uint8_t*>(d_queries);
    a.qf = qf;
    a.Q = (int)Q;
    a.k = k;
    a.ngran = (N + kSelRows - 1) / kSelRows;
    a.out_ids = d_out_ids;
    a.out_lcp = d_out_lcp;
    a.status = lib_status_word();
    a.plane = nullptr;
    a.sorted = Q >= kSelSortedMinQ ? 1 : 0;
    Carver cv;
    // zeroed together: hist, n2, n4
    cv.add(&a.hist, (size_t)Q * (L + 1));
    cv.add(&a.n2, (size_t)Q);
    cv.add(&a.n4, (size_t)Q);
    cv.add(&a.cnt, (size_t)Q * a.ngran);
    cv.add(&a.list2, (size_t)Q * kSelList);
    cv.add(&a.list4, (size_t)Q * kSelList);
    cv.add(&a.plane, (size_t)N);  // the walks read word 0 from L2 instead of the rows
    void* base = nullptr;
    LCP_CUDA_TRY(cv.alloc(&base, s));
    cudaError_t e =
        cudaMemsetAsync(a.hist, 0, (size_t)(reinterpret_cast<char*>(a.n4 + Q) - reinterpret_cast<char*>(a.hist)), s);
    CUtensorMap tm;
    memset(&tm, 0, sizeof(tm));
    const int use_tma = sel_tensor_map(d_tokens, N, f, &tm) ? 1 : 0;
    const SelSetup* su = e == cudaSuccess ? sel_setup() : nullptr;
    if (e == cudaSuccess && !su) e = cudaErrorUnknown;
    if (e == cudaSuccess) {
        // one wave of count CTAs (each warp walks its tiles through its ring)
        const int warps = kSelCountWarps;
        a.stages = kSelWarpStages;
        const int64_t ctas = (int64_t)sm_count() * su->count_ctas[f.tb == 2 ? 1 : 0];
        const int64_t want = (a.ngran + warps - 1) / warps;
        const unsigned grid = (unsigned)(want < ctas ? want : ctas);
        const size_t count_smem = sel_count_smem((int)Q, warps, a.stages);
        if (f.tb == 2)
            LCP_TIMED_LAUNCH(k_sel_count<2>, grid, warps * 32, count_smem, s, tm, a, use_tma);
        else
            LCP_TIMED_LAUNCH(k_sel_count<1>, grid, warps * 32, count_smem, s, tm, a, use_tma);
        const int64_t sms = sm_count();
        const int athr = Q <= 2 * sms ? kSelAnswerWide : (Q <= 3 * sms ? kSelAnswerMid : kSelAnswerNarrow);
        LCP_TIMED_LAUNCH(k_sel_answer, (unsigned)Q, athr, sel_answer_smem(k), s, a);
    }
    const cudaError_t fe = cudaFreeAsync(base, s);
    if (e == cudaSuccess) e = fe;
    return e == cudaSuccess ? LCP_OK : cuda_status(e);
}

}  // namespace lcph
