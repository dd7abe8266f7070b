// Index build: Algorithm 1 (BuildLCPIndex) + Algorithm 2 in array form.
//
// 1. Keys: word 0 of every row with its id (the load asks L2 for 64 bytes:
//    only 8 bytes of each row are needed here).
// 2. A stable LSD radix sort of the (word 0, id) pairs: 8-bit digits,
//    reduce-then-scan passes (sort.cu), as two 32-bit sorts -- the low half
//    of word 0, then the high half gathered by id -- so that every pass
//    moves 8-byte (key, id) pairs.
// 3. Rows sharing word 0 with another row form tie groups, found straight
//    from the equality flags of the sorted keys: a group of at most 32 rows
//    is ranked by a warp, one of 33-2048 rows by a CTA, on word 1 and -- only
//    for rows tied there -- the later words, then the id.  Groups of more
//    than 2048 rows, or with a row tied on word 1 with more than 64 others (heavy
//    duplication; none on the paper's workloads) take
//    the exact refinement instead: round r sorts the still-tied rows by
//    (tie group, word r), a stable LSD sort on word r followed by one on the
//    group rank, until every prefix is unique.
// 4. The rows are gathered into sorted order with their heads and H, the LCP
//    of each row with the one before it (Algorithm 2's subtree sizes become
//    LCP intervals of H).
// 5. The search's tables: pos, the depth-1 buckets, the min tree over H, the
//    sorted 128-row blocks and the sparse table of their K smallest ids (on
//    two stream branches), then the heavy trie nodes' tie lists (tielists.cu).
// Every pass is stable, so equal rows stay in id order: the posting-list
// order of Algorithm 1.
#include "search.cuh"
#include "sort.cuh"

namespace lcpk {

// Word 0 of every row, in halves: the low half twice (the sort's key, and a
// copy by id for the equality test), the high half by id, and vals[i] = i.
// Only the first 8 bytes of each row are needed, so the aligned load asks L2
// for a 64-byte fetch rather than a whole line.
__global__ void k_keys_word0(const uint8_t* __restrict__ tokens, RowFmt f, uint32_t n,
                             uint32_t* __restrict__ key_lo, uint32_t* __restrict__ lo_by_id,
                             uint32_t* __restrict__ hi_by_id, uint32_t* __restrict__ vals) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint8_t* row = row_of(tokens, i, f);
    uint64_t x;
    if (f.aligned8) {
        asm("ld.global.nc.L2::64B.u64 %0, [%1];" : "=l"(x) : "l"(row));
        x = msb_first(x, f.tb);
    } else {
        x = pack_word(row, 0, f);
    }
    key_lo[i] = (uint32_t)x;
    lo_by_id[i] = (uint32_t)x;
    hi_by_id[i] = (uint32_t)(x >> 32);
    vals[i] = i;
}

// The sorted ids, and eq[i] = 1 where the row at sorted position i has the
// same word 0 as the row before it (high halves in sorted order, low halves
// by id).
__global__ void k_ids_eq(const uint32_t* __restrict__ vs, const uint32_t* __restrict__ key_hi,
                         const uint32_t* __restrict__ lo_by_id, uint32_t n, int32_t* __restrict__ ids,
                         uint8_t* __restrict__ eq) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t v = vs[i];
    ids[i] = (int32_t)v;
    bool e = false;
    if (i > 0 && key_hi[i] == key_hi[i - 1]) {
        const uint32_t u = vs[i - 1];
        e = v < n && u < n && lo_by_id[v] == lo_by_id[u];
    }
    eq[i] = e ? 1 : 0;
}

// keys[i] = word r of the row at sorted position act[i]; vals[i] = i.
__global__ void k_keys_active(const uint8_t* __restrict__ tokens, RowFmt f, uint32_t n_rows,
                              const int32_t* __restrict__ ids, const uint32_t* __restrict__ act,
                              uint32_t m, int r, uint64_t* __restrict__ keys,
                              uint32_t* __restrict__ vals) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int32_t id = ids[act[i]];
    keys[i] = (uint32_t)id < n_rows ? pack_word(row_of(tokens, id, f), r, f) : 0ull;
    vals[i] = i;
}

// After the word sort: key by index (for the tie test) and group keys.
__global__ void k_group_keys(const uint64_t* __restrict__ ks, const uint32_t* __restrict__ vs,
                             const uint32_t* __restrict__ grp, uint32_t m,
                             uint64_t* __restrict__ kbi, uint32_t* __restrict__ gk,
                             uint32_t* __restrict__ gv) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    uint32_t v = vs[i];
    kbi[v] = ks[i];
    gk[i] = grp[v];
    gv[i] = v;
}

__global__ void k_apply_gather(const uint32_t* __restrict__ fv, const int32_t* __restrict__ ids,
                               const uint32_t* __restrict__ act, const uint64_t* __restrict__ kbi,
                               const uint32_t* __restrict__ grp, uint32_t m,
                               int32_t* __restrict__ newid, uint64_t* __restrict__ fkey,
                               uint32_t* __restrict__ fgrp) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    uint32_t v = fv[i];
    newid[i] = ids[act[v]];
    fkey[i] = kbi[v];
    fgrp[i] = grp[v];
}

__global__ void k_apply_scatter(const int32_t* __restrict__ newid, const uint32_t* __restrict__ act,
                                const uint64_t* __restrict__ fkey,
                                const uint32_t* __restrict__ fgrp, uint32_t m,
                                int32_t* __restrict__ ids, uint8_t* __restrict__ eq) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    ids[act[i]] = newid[i];
    eq[i] = (i > 0 && fgrp[i] == fgrp[i - 1] && fkey[i] == fkey[i - 1]) ? 1 : 0;
}

__global__ void k_remap_active(const uint32_t* __restrict__ act, const uint32_t* __restrict__ idx,
                               uint32_t m, uint32_t* __restrict__ act2) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    act2[j] = act[idx[j]];
}

// Lexicographic comparison of two raw rows from word w0 on, then by id.
__device__ __forceinline__ bool row_less(const uint8_t* __restrict__ tokens, const RowFmt& f, int w0,
                                         int32_t a, int32_t b) {
    const uint8_t* ra = row_of(tokens, a, f);
    const uint8_t* rb = row_of(tokens, b, f);
    for (int w = w0; w < f.W; ++w) {
        const uint64_t x = pack_word(ra, w, f), y = pack_word(rb, w, f);
        if (x != y) return x < y;
    }
    return a < b;
}

// Orders two rows of one tie group: by word 1 (given), then the later words,
// then id.  Word 0 is equal inside a group.
__device__ __forceinline__ bool tie_less(const uint8_t* __restrict__ tokens, const RowFmt& f,
                                         uint64_t ka, int32_t a, uint64_t kb, int32_t b) {
    if (ka != kb) return ka < kb;
    return row_less(tokens, f, 2, a, b);  // rare: equal on word 1 too
}

constexpr uint32_t kMidMax = 2048;  // largest tie group ranked by one CTA

// Rows tied on word 0, found straight from eq: a warp takes 32 consecutive
// sorted positions and handles each tie group that starts among them.  A
// group of at most 32 rows is ranked in registers (word 1 loaded once per row,
// shuffles; later words and then ids only for rows tied on word 1) and
// written back in order; groups of 33..kMidMax rows are listed for
// k_group_sort_mid; the rows of larger groups are counted for the exact
// refinement.
__global__ void __launch_bounds__(256) k_group_scan_sort(const uint8_t* __restrict__ tokens, RowFmt f,
                                                         const uint8_t* __restrict__ eq, uint32_t n,
                                                         int32_t* __restrict__ ids,
                                                         uint32_t* __restrict__ big_start,
                                                         uint32_t* __restrict__ big_len,
                                                         uint32_t* __restrict__ big_count,
                                                         uint32_t* __restrict__ huge_count) {
    const unsigned lane = lane_id();
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); (uint64_t)c * 32 < n; c += nwarps) {
        const uint32_t p = c * 32 + lane;
        const bool first = p < n && !eq[p] && p + 1 < n && eq[p + 1];  // first row of a tie group
        unsigned starts = __ballot_sync(0xffffffffu, first);
        while (starts) {
            const uint32_t gs = c * 32 + (uint32_t)(__ffs(starts) - 1);
            starts &= starts - 1;
            uint32_t len = 1;  // rows gs+1, gs+2, ... while eq holds
            for (uint32_t q = gs + 1;; q += 32) {
                const uint32_t t = q + lane;
                const unsigned brk = __ballot_sync(0xffffffffu, !(t < n && eq[t]));
                if (brk) {
                    len += (uint32_t)(__ffs(brk) - 1);
                    break;
                }
                len += 32;
            }
            if (len > 32) {
                if (lane == 0) {
                    if (len <= kMidMax) {
                        const uint32_t b = atomicAdd(big_count, 1u);
                        big_start[b] = gs;
                        big_len[b] = len;
                    } else {
                        atomicAdd(huge_count, len);
                    }
                }
                continue;
            }
            const int32_t my = lane < len ? ids[gs + lane] : 0;
            const uint64_t key = lane < len ? pack_word(row_of(tokens, my, f), 1, f) : 0ull;
            uint32_t rank = 0;
            for (uint32_t j = 0; j < len; ++j) {
                const int32_t oid = __shfl_sync(0xffffffffu, my, j);
                const uint64_t ok = __shfl_sync(0xffffffffu, key, j);
                if (lane < len && j != lane && tie_less(tokens, f, ok, oid, key, my)) ++rank;
            }
            __syncwarp();
            if (lane < len) ids[gs + rank] = my;
            __syncwarp();
        }
    }
}

// Groups of 33..kMidMax rows: one CTA of 1024 threads, a row per thread (two
// past 1024 rows), word-1 keys staged in shared memory.  Each row's rank is a
// branch-free count of the keys below its own; a row whose word 1 is shared
// with others compares the later words of those rows, then the ids.  If some
// row shares word 1 with more than kMidTied others, the group is left to the
// exact refinement (its rows are counted into huge_count), which keeps the
// row comparisons of a group bounded.
constexpr uint32_t kMidTied = 64;

__global__ void __launch_bounds__(1024, 1) k_group_sort_mid(const uint8_t* __restrict__ tokens, RowFmt f,
                                                         int32_t* __restrict__ ids,
                                                         const uint32_t* __restrict__ big_start,
                                                         const uint32_t* __restrict__ big_len,
                                                         const uint32_t* __restrict__ big_count,
                                                         uint32_t* __restrict__ huge_count) {
    __shared__ int32_t sid[kMidMax];
    __shared__ uint64_t skey[kMidMax];
    const uint32_t nbig = *big_count;
    const uint32_t t = threadIdx.x;
    for (uint32_t b = blockIdx.x; b < nbig; b += gridDim.x) {  // CTA per group
        const uint32_t gs = big_start[b], n = big_len[b];
        for (uint32_t i = t; i < n; i += 1024) {
            const int32_t id = ids[gs + i];
            sid[i] = id;
            skey[i] = pack_word(row_of(tokens, id, f), 1, f);
        }
        __syncthreads();
        auto count_below = [&](uint32_t i, uint32_t& tied) -> uint32_t {
            const uint64_t ki = skey[i];
            uint32_t rank = 0;
            tied = 0;
#pragma unroll 8
            for (uint32_t j = 0; j < n; ++j) {
                const uint64_t kj = skey[j];
                rank += kj < ki;
                tied += kj == ki;
            }
            return rank;
        };
        auto tied_below = [&](uint32_t i) -> uint32_t {  // rows equal on word 1 ordered before row i
            const uint64_t ki = skey[i];
            const int32_t my = sid[i];
            uint32_t r = 0;
            for (uint32_t j = 0; j < n; ++j)
                if (j != i && skey[j] == ki && row_less(tokens, f, 2, sid[j], my)) ++r;
            return r;
        };
        uint32_t r0 = 0, r1 = 0, t0 = 0, t1 = 0;
        if (t < n) r0 = count_below(t, t0);
        if (t + 1024 < n) r1 = count_below(t + 1024, t1);
        if (__syncthreads_or(t0 > kMidTied + 1 || t1 > kMidTied + 1)) {  // (counts include the row itself)
            if (t == 0) atomicAdd(huge_count, n);
        } else {
            if (t0 > 1) r0 += tied_below(t);
            if (t1 > 1) r1 += tied_below(t + 1024);
            __syncthreads();
            if (t < n) ids[gs + r0] = sid[t];
            if (t + 1024 < n) ids[gs + r1] = sid[t + 1024];
        }
        __syncthreads();  // the shared arrays are refilled for the next group
    }
}

// rows[p][w] = packed word w of raw row ids[p]; head[p] = rows[p][0].
__global__ void k_gather_rows(const uint8_t* __restrict__ tokens, RowFmt f, int64_t n,
                              const int32_t* __restrict__ ids, uint64_t* __restrict__ rows,
                              uint64_t* __restrict__ head) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t total = n * f.W;
    if (e >= total) return;
    int64_t p = e / f.W;
    int w = (int)(e - p * f.W);
    int32_t id = ids[p];
    uint64_t x = (uint64_t)id < (uint64_t)n ? pack_word(row_of(tokens, id, f), w, f) : 0ull;
    rows[e] = x;
    if (w == 0) head[p] = x;
}

// Same with two words per thread and 16-byte accesses (rows of an even number
// of words, 16-byte aligned raw rows and output).
__global__ void k_gather_rows_v2(const uint8_t* __restrict__ tokens, RowFmt f, int64_t n,
                                 const int32_t* __restrict__ ids, uint64_t* __restrict__ rows,
                                 uint64_t* __restrict__ head) {
    const int half = f.W >> 1;
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * half) return;
    const int64_t p = e / half;
    const int h = (int)(e - p * half);
    const int32_t id = ids[p];
    ulonglong2 v = make_ulonglong2(0ull, 0ull);
    if ((uint64_t)id < (uint64_t)n) {
        const ulonglong2 raw = __ldg(reinterpret_cast<const ulonglong2*>(row_of(tokens, id, f)) + h);
        v.x = msb_first(raw.x, f.tb);
        v.y = msb_first(raw.y, f.tb);
    }
    reinterpret_cast<ulonglong2*>(rows)[e] = v;
    if (h == 0) head[p] = v.x;
}

// Rows into sorted order together with head and H, for rows of W words with
// W / 2 dividing 32 (16-byte aligned raw rows and output).  A warp owns
// kGatherSteps * (64 / W) consecutive sorted positions, 32 / (W / 2) rows per
// step with two words per lane; all steps' loads are issued before any compare.
// The previous row's words come from the lanes one row below (a shuffle) --
// only the row before the warp's first one is loaded again -- and a row's
// LCP with its predecessor is the minimum over its lanes of the first
// difference in their two words.
constexpr int kGatherSteps = 2;

// Words 2h, 2h+1 of the row at sorted position p (zeros off the ends).
__device__ __forceinline__ ulonglong2 gather_half_words(const uint8_t* __restrict__ tokens, const RowFmt& f,
                                                        int64_t n, const int32_t* __restrict__ ids, int64_t p,
                                                        int h) {
    ulonglong2 v = make_ulonglong2(0ull, 0ull);
    if (p >= 0 && p < n) {
        const int32_t id = ids[p];
        if ((uint64_t)id < (uint64_t)n) {
            const ulonglong2 raw = __ldg(reinterpret_cast<const ulonglong2*>(row_of(tokens, id, f)) + h);
            v.x = msb_first(raw.x, f.tb);
            v.y = msb_first(raw.y, f.tb);
        }
    }
    return v;
}

__global__ void __launch_bounds__(256) k_gather_rows_lcp(const uint8_t* __restrict__ tokens, RowFmt f, int64_t n,
                                                         const int32_t* __restrict__ ids,
                                                         uint64_t* __restrict__ rows, uint64_t* __restrict__ head,
                                                         uint8_t* __restrict__ H) {
    const int half = f.W >> 1;  // a power of two <= 32
    const int lg = __ffs(half) - 1;
    const int R = 32 >> lg;  // rows per step
    const unsigned lane = lane_id();
    const int rl = (int)(lane >> lg), h = (int)(lane & (half - 1));
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t p0 = warp * (int64_t)(R * kGatherSteps);
    if (p0 >= n) return;  // warp-uniform
    ulonglong2 v[kGatherSteps];
#pragma unroll
    for (int j = 0; j < kGatherSteps; ++j) v[j] = gather_half_words(tokens, f, n, ids, p0 + (int64_t)j * R + rl, h);
    // the row before the first one, held where a step's last row would be
    ulonglong2 last = rl == R - 1 ? gather_half_words(tokens, f, n, ids, p0 - 1, h) : make_ulonglong2(0ull, 0ull);
    constexpr int kNone = 1 << 20;
#pragma unroll
    for (int j = 0; j < kGatherSteps; ++j) {
        const ulonglong2 cur = v[j];
        const uint64_t ux = __shfl_up_sync(0xffffffffu, cur.x, half);
        const uint64_t uy = __shfl_up_sync(0xffffffffu, cur.y, half);
        const uint64_t lx = __shfl_sync(0xffffffffu, last.x, (int)lane + 32 - half);
        const uint64_t ly = __shfl_sync(0xffffffffu, last.y, (int)lane + 32 - half);
        const uint64_t ax = rl > 0 ? ux : lx, ay = rl > 0 ? uy : ly;
        const uint64_t x0 = ax ^ cur.x, x1 = ay ^ cur.y;
        int l = x0 ? (2 * h) * f.tpw + __clzll((long long)x0) / f.bits
                   : (x1 ? (2 * h + 1) * f.tpw + __clzll((long long)x1) / f.bits : kNone);
        for (int o = 1; o < half; o <<= 1) l = min(l, __shfl_xor_sync(0xffffffffu, l, o));
        const int64_t p = p0 + (int64_t)j * R + rl;
        if (p < n) {
            reinterpret_cast<ulonglong2*>(rows)[p * half + h] = cur;
            if (h == 0) {
                head[p] = cur.x;
                H[p] = p == 0 ? (uint8_t)0 : (uint8_t)min(l, min(f.L, 255));  // 255: wide rows
            }
        }
        last = cur;
    }
}

// H[p] = LCP(rows[p-1], rows[p]), H[0] = 0.
__global__ void k_adjacent_lcp(const uint64_t* __restrict__ rows, int64_t n, int W, int L, int tpw,
                               int bits, uint8_t* __restrict__ H) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    if (p == 0) {
        H[0] = 0;
        return;
    }
    const uint64_t* a = rows + (p - 1) * W;
    const uint64_t* b = rows + p * W;
    int l = L;
    for (int w = 0; w < W; ++w) {
        uint64_t x = a[w] ^ b[w];
        if (x) {
            l = w * tpw + (__clzll((long long)x) / bits);
            if (l > L) l = L;
            break;
        }
    }
    H[p] = (uint8_t)min(l, 255);  // rows longer than 255 tokens keep H clamped (unused there)
}

__global__ void k_inverse(const int32_t* __restrict__ ids, int64_t n, int32_t* __restrict__ pos) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) {
        int32_t id = ids[p];
        if ((uint64_t)id < (uint64_t)n) pos[id] = (int32_t)p;
    }
}

// out[b] = min(in[32b .. 32b+31]) (entries past n_in ignored).
__global__ void k_min32(const uint8_t* __restrict__ in, int64_t n_in, uint8_t* __restrict__ out,
                        int64_t n_out) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_out) return;
    int64_t s = b * 32, e = s + 32 < n_in ? s + 32 : n_in;
    uint32_t m = 255;
    for (int64_t i = s; i < e; ++i) m = min(m, (uint32_t)in[i]);
    out[b] = (uint8_t)m;
}

constexpr int kAuxThreads = 1024;
constexpr int64_t kTreeChunk = 32768;  // H entries per tree CTA: 1024 x 32

struct AuxArgs {
    const uint8_t* H;
    int64_t N;
    uint8_t* hmin;
    int lev;              // tree levels written here (<= 3)
    int64_t hoff[3], hlen[3];
    unsigned tree_ctas;
    const int32_t* ids;
    int64_t nblk;
    uint32_t* sblk;
    uint8_t* soff;
};

// Minimum of the 32 H entries starting at s (entries past n count as 255).
__device__ __forceinline__ uint32_t min32_bytes(const uint8_t* __restrict__ H, int64_t s, int64_t n) {
    if (s + 32 <= n) {
        const uint4 a = *reinterpret_cast<const uint4*>(H + s);
        const uint4 b = *reinterpret_cast<const uint4*>(H + s + 16);
        uint32_t m = __vminu4(__vminu4(__vminu4(a.x, a.y), __vminu4(a.z, a.w)),
                              __vminu4(__vminu4(b.x, b.y), __vminu4(b.z, b.w)));
        m = __vminu4(m, m >> 16);
        m = __vminu4(m, m >> 8);
        return m & 255u;
    }
    uint32_t m = 255;
    for (int64_t i = s; i < n && i < s + 32; ++i) m = min(m, (uint32_t)H[i]);
    return m;
}

// CTAs below tree_ctas: levels 1..3 of the min tree for 32768 consecutive H
// entries (thread -> level-1 entry, warp -> level 2, CTA -> level 3).  The
// rest: one warp per 128-position block, its (id, offset) pairs sorted
// ascending with the register bitonic network (padding 0xFFFFFFFF).
__global__ void __launch_bounds__(kAuxThreads) k_aux_tree_blocks(AuxArgs a) {
    const int lane = (int)lane_id(), warp = threadIdx.x >> 5;
    if (blockIdx.x < a.tree_ctas) {
        __shared__ uint32_t wmin[kAuxThreads / 32];
        const int64_t e1 = (int64_t)blockIdx.x * kAuxThreads + threadIdx.x;  // level-1 entry
        const uint32_t m1 = e1 < a.hlen[0] ? min32_bytes(a.H, e1 * 32, a.N) : 255u;
        if (e1 < a.hlen[0]) a.hmin[a.hoff[0] + e1] = (uint8_t)m1;
        if (a.lev < 2) return;
        const uint32_t m2 = __reduce_min_sync(0xffffffffu, m1);
        const int64_t e2 = (int64_t)blockIdx.x * 32 + warp;
        if (lane == 0) {
            if (e2 < a.hlen[1]) a.hmin[a.hoff[1] + e2] = (uint8_t)m2;
            wmin[warp] = m2;
        }
        if (a.lev < 3) return;
        __syncthreads();
        if (warp == 0) {
            const uint32_t m3 = __reduce_min_sync(0xffffffffu, wmin[lane]);
            if (lane == 0 && (int64_t)blockIdx.x < a.hlen[2]) a.hmin[a.hoff[2] + blockIdx.x] = (uint8_t)m3;
        }
        return;
    }
    const int64_t b = (int64_t)(blockIdx.x - a.tree_ctas) * (kAuxThreads / 32) + warp;
    if (b >= a.nblk) return;
    uint64_t v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int off = lane * 4 + e;
        const int64_t p = b * kBlk + off;
        v[e] = p < a.N ? (((uint64_t)(uint32_t)a.ids[p] << 8) | (uint64_t)off) : ~0ull;
    }
    warp_bitonic<4, uint64_t>(v);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int t = lane * 4 + e;
        a.sblk[b * kBlk + t] = v[e] == ~0ull ? kInf : (uint32_t)(v[e] >> 8);
        a.soff[b * kBlk + t] = (uint8_t)(v[e] & 255u);
    }
}

// The search's top levels: top[j] = head[j * n / T] for j < T.
__global__ void k_top_sample(const uint64_t* __restrict__ head, int64_t n, int T, uint64_t* __restrict__ top) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < T) top[j] = head[(int64_t)j * n / T];
}

// Depth-1 buckets: bkt[t] = first sorted position whose first token is >= t,
// for t in [0, 2^bits] (bkt[2^bits] = n): one binary search on head per token.
__global__ void k_buckets(const uint64_t* __restrict__ head, int64_t n, int bits,
                          int32_t* __restrict__ bkt) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t ntok = 1ll << bits;
    if (t > ntok) return;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)(head[mid] >> (64 - bits)) < t) lo = mid + 1;
        else hi = mid;
    }
    bkt[t] = (int32_t)lo;
}

// Depth-2 bucket tables.  k_sub_assign: the first tokens whose depth-1
// bucket holds at least kSub2Min rows get a table each (numbered by an
// atomic counter, at most kSub2Max; which buckets get one when there are
// more is not fixed, and answers never depend on it).  k_sub_mark: the first
// and the last row of each (first, second token) run in such a bucket write
// the run's start and end at its second token; entries of second tokens
// that do not occur are never read (a search reads the run of a neighbour
// row's first two tokens).
__global__ void k_sub_assign(const int32_t* __restrict__ bkt, int bits, int32_t* __restrict__ sub_idx,
                             uint32_t* __restrict__ count) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= (1 << bits)) return;
    int32_t t = -1;
    if (bkt[v + 1] - bkt[v] >= kSub2Min) {
        const uint32_t r = atomicAdd(count, 1u);
        if (r < (uint32_t)kSub2Max) t = (int32_t)r;
    }
    sub_idx[v] = t;
}

__global__ void k_sub_mark(const uint64_t* __restrict__ head, int64_t n, int bits, const int32_t* __restrict__ sub_idx,
                           int2* __restrict__ sub) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint64_t h = head[p];
    const int32_t si = sub_idx[h >> (64 - bits)];
    if (si < 0) return;
    const uint64_t m2 = ~0ull << (64 - 2 * bits);  // the first two tokens
    const uint32_t t1 = (uint32_t)(h >> (64 - 2 * bits)) & ((1u << bits) - 1);
    int2* e = sub + ((int64_t)si << bits) + t1;
    if (p == 0 || ((head[p - 1] ^ h) & m2) != 0) e->x = (int32_t)p;
    if (p == n - 1 || ((head[p + 1] ^ h) & m2) != 0) e->y = (int32_t)(p + 1);
}

// First K entries of the merge of the sorted K-lists A and B (smem) into O
// (smem or global); lane l writes entries [l*K/32, (l+1)*K/32) by merge path.
__device__ __forceinline__ void merge_k(const uint32_t* A, const uint32_t* B, uint32_t* O, int K, int lane) {
    const int per = K / 32;
    const int d0 = lane * per;
    int lo = d0 - K > 0 ? d0 - K : 0, hi = d0 < K ? d0 : K;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (A[mid] <= B[d0 - 1 - mid]) lo = mid + 1;
        else hi = mid;
    }
    int i = lo, j = d0 - lo;
    for (int t = 0; t < per; ++t) {
        const bool takeA = (i < K) && (j >= K || A[i] <= B[j]);
        O[d0 + t] = takeA ? A[i++] : B[j++];
    }
}

// The K = 32E smallest of two ascending lists a, b of K ids (lane l holds
// entries lE .. lE+E-1 of each), ascending, into a: the minimum of a and b
// reversed is a bitonic sequence holding the K smallest, which the bitonic
// half-cleaners then sort, all in registers.
template <int E>
__device__ __forceinline__ void st_merge_regs(uint32_t (&a)[E], const uint32_t (&b)[E], unsigned lane) {
#pragma unroll
    for (int e = 0; e < E; ++e) a[e] = min(a[e], __shfl_sync(0xffffffffu, b[E - 1 - e], 31 - (int)lane));
#pragma unroll
    for (int st = 16 * E; st >= 1; st >>= 1) {
        if (st >= E) {
            const int m = st / E;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const uint32_t o = __shfl_xor_sync(0xffffffffu, a[e], m);
                a[e] = (lane & (unsigned)m) ? max(a[e], o) : min(a[e], o);
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                if ((e & st) == 0) {
                    const uint32_t lo = min(a[e], a[e + st]), hi = max(a[e], a[e + st]);
                    a[e] = lo;
                    a[e + st] = hi;
                }
            }
        }
    }
}

template <int E>
__device__ __forceinline__ void st_load(const uint32_t* __restrict__ p, uint32_t (&v)[E]) {
    if constexpr (E == 1) {
        v[0] = __ldg(p);
    } else if constexpr (E == 2) {
        const uint2 x = __ldg(reinterpret_cast<const uint2*>(p));
        v[0] = x.x;
        v[1] = x.y;
    } else {
#pragma unroll
        for (int e = 0; e < E; e += 4) {
            const uint4 x = __ldg(reinterpret_cast<const uint4*>(p + e));
            v[e] = x.x;
            v[e + 1] = x.y;
            v[e + 2] = x.z;
            v[e + 3] = x.w;
        }
    }
}

template <int E>
__device__ __forceinline__ void st_store(uint32_t* __restrict__ p, const uint32_t (&v)[E]) {
    if constexpr (E == 1) {
        p[0] = v[0];
    } else if constexpr (E == 2) {
        *reinterpret_cast<uint2*>(p) = make_uint2(v[0], v[1]);
    } else {
#pragma unroll
        for (int e = 0; e < E; e += 4) *reinterpret_cast<uint4*>(p + e) = make_uint4(v[e], v[e + 1], v[e + 2], v[e + 3]);
    }
}

// Sparse-table levels j .. j+g-1 (g <= G) for K = 32E in one launch, merged
// in registers.  Level j+r at i is the K smallest of level j-1 at
// i + m*half for m < 2^(r+1): a warp loads those 2^G lists of its start
// block and merges them pairwise up the tree, writing the tree's left spine
// (levels j .. j+g-1 at i).  Spines of other start blocks are recomputed,
// not shared: 2^G - 1 merges for g levels and g - 1 fewer launches.  P start
// blocks per warp, all loads issued before any merge.
constexpr int kStRegsMaxG = 4;  // levels per launch of the register merge, at most

struct StValid {
    int64_t v[kStRegsMaxG];  // start blocks of each level of the launch
};

template <int E, int G, int P>
__global__ void __launch_bounds__(256) k_st_levels_regs(const uint32_t* __restrict__ prev, int64_t prev_stride,
                                                        int64_t prev_valid, int64_t half, int g,
                                                        int64_t level_stride, StValid vb,
                                                        uint32_t* __restrict__ out0) {
    static_assert(G <= kStRegsMaxG, "levels per launch");
    constexpr int K = 32 * E, M = 1 << G;
    const unsigned lane = lane_id();
    const int64_t i0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * P;
    const int64_t valid0 = vb.v[0];
    if (i0 >= valid0) return;  // warp-uniform
    uint32_t v[P][M][E];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int64_t i = i0 + q;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int64_t pos = i + m * half;
            // entries past the previous level only feed spine levels that
            // are not stored
            if (i < valid0 && m < (2 << (g - 1)) && pos < prev_valid) {
                st_load<E>(prev + pos * prev_stride + lane * E, v[q][m]);
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) v[q][m][e] = kInf;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int64_t i = i0 + q;
#pragma unroll
        for (int r = 0; r < G; ++r) {
#pragma unroll
            for (int m = 0; m < (M >> (r + 1)); ++m) {
                uint32_t t[E];
#pragma unroll
                for (int e = 0; e < E; ++e) t[e] = v[q][2 * m][e];
                st_merge_regs<E>(t, v[q][2 * m + 1], lane);
#pragma unroll
                for (int e = 0; e < E; ++e) v[q][m][e] = t[e];
            }
            if (r < g && i < vb.v[r]) st_store<E>(out0 + r * level_stride + i * K + lane * E, v[q][0]);
        }
    }
}

// Levels per launch and start blocks per warp of the register merge, by E.
template <int E>
struct StRegsShape;
template <>
struct StRegsShape<1> {
    static constexpr int G = 3, P = 1;
};
template <>
struct StRegsShape<2> {
    static constexpr int G = 2, P = 2;
};
template <>
struct StRegsShape<4> {
    static constexpr int G = 2, P = 2;
};

constexpr int kStMaxGroup = 3;  // sparse-table levels per launch (K <= 32)

// Sparse-table levels j .. j+g-1 in one launch, one warp per start block i.
// Level j+r at i is the K smallest of level j-1 at i + m*half for
// m < 2^(r+1) (disjoint position spans, so no duplicates): the warp merges
// those lists pairwise up the tree and writes the tree's left spine, which
// is exactly levels j .. j+g-1 at i.  Lists of other warps' spines are
// recomputed rather than waited for (2^g - 1 merges instead of g), trading
// a little arithmetic for g - 1 fewer launches.
__global__ void __launch_bounds__(256) k_st_levels(const uint32_t* __restrict__ prev, int64_t prev_stride,
                                                   int64_t half, int g, int K, int64_t level_stride,
                                                   int64_t valid0, int64_t valid1, int64_t valid2,
                                                   uint32_t* __restrict__ out0) {
    extern __shared__ uint32_t st_smem[];
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= valid0) return;
    uint32_t* base = st_smem + (size_t)(threadIdx.x >> 5) * (g > 1 ? 6 : 3) * K;
    uint32_t *A = base, *B = base + K, *S0 = base + 2 * K, *S1 = base + 3 * K, *T0 = base + 4 * K,
             *T1 = base + 5 * K;
    // level j at i + m*2*half, m = 0 .. 3: merge of prev lists (2m, 2m+1)
    auto pair = [&](int64_t m, uint32_t* dst) {
        const uint32_t* ga = prev + (i + 2 * m * half) * prev_stride;
        const uint32_t* gb = prev + (i + (2 * m + 1) * half) * prev_stride;
        for (int t = lane; t < K; t += 32) {
            A[t] = ga[t];
            B[t] = gb[t];
        }
        __syncwarp();
        merge_k(A, B, dst, K, lane);
        __syncwarp();
    };
    pair(0, S0);
    for (int t = lane; t < K; t += 32) out0[i * K + t] = S0[t];
    if (g < 2 || i >= valid1) return;
    pair(1, S1);
    merge_k(S0, S1, T0, K, lane);  // level j+1 at i
    __syncwarp();
    for (int t = lane; t < K; t += 32) out0[level_stride + i * K + t] = T0[t];
    if (g < 3 || i >= valid2) return;
    pair(2, S0);
    pair(3, S1);
    merge_k(S0, S1, T1, K, lane);  // level j+1 at i + 4*half
    __syncwarp();
    merge_k(T0, T1, S0, K, lane);  // level j+2 at i
    __syncwarp();
    for (int t = lane; t < K; t += 32) out0[2 * level_stride + i * K + t] = S0[t];
}

}  // namespace lcpk

namespace lcph {
using namespace lcpk;

static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// The build's scratch arrays, carved from one block.
struct BuildScratch {
    uint64_t *k0, *k1, *kbi, *fkey;
    uint32_t *v0, *v1, *act, *grp, *act2, *grp2, *idx2, *gk, *gv, *gk1, *gv1, *fgrp;
    int32_t* newid;
    uint8_t* eq;
    void carve(Carver& c, uint32_t N) {
        for (uint64_t** p : {&k0, &k1, &kbi, &fkey}) c.add(p, N);
        for (uint32_t** p : {&v0, &v1, &act, &grp, &act2, &grp2, &idx2, &gk, &gv, &gk1, &gv1, &fgrp}) c.add(p, N);
        c.add(&newid, N);
        c.add(&eq, N);
    }
};

size_t build_scratch_bytes(int64_t N64) {
    const uint32_t N = (uint32_t)(N64 > 1 ? N64 : 2);
    BuildScratch b;
    Carver c;
    b.carve(c, N);
    return c.total + sort_work_bytes(N);
}

int build_sorted_ids(const void* tokens, const RowFmt& f, int64_t N64, int32_t* ids_out, int* err,
                     cudaStream_t s, uint32_t* huge_host, void* scratch) {
    if (N64 <= 0) return LCP_OK;
    uint32_t N = (uint32_t)N64;
    const uint8_t* tk = reinterpret_cast<const uint8_t*>(tokens);
    if (N == 1) {
        LCP_CUDA_TRY(cudaMemsetAsync(ids_out, 0, sizeof(int32_t), s));
        return LCP_OK;
    }
    // scratch: one block, allocated here unless the caller provides it
    BuildScratch b;
    Carver c;
    b.carve(c, N);
    void* arena = nullptr;
    SortWork w;
    int rc;
    if (scratch) {
        c.place(scratch);
        rc = sort_work_place(w, N, err, static_cast<char*>(scratch) + c.total);
    } else {
        LCP_CUDA_TRY(c.alloc(&arena, s));
        rc = sort_work_alloc(w, N, err, s);
    }
    uint64_t *k0 = b.k0, *k1 = b.k1, *kbi = b.kbi, *fkey = b.fkey;
    uint32_t *v0 = b.v0, *v1 = b.v1, *act = b.act, *grp = b.grp, *act2 = b.act2, *grp2 = b.grp2, *idx2 = b.idx2;
    uint32_t *gk = b.gk, *gv = b.gv, *gk1 = b.gk1, *gv1 = b.gv1, *fgrp = b.fgrp;
    int32_t* newid = b.newid;
    uint8_t* eq = b.eq;
    auto cleanup = [&]() {
        if (arena) cudaFreeAsync(arena, s);
        if (w.arena) sort_work_free(w, s);
    };
    if (rc) {
        cleanup();
        return rc;
    }
    // first sort key: (word 0, id) over all rows, as two stable 32-bit LSD
    // sorts -- the low half, then the high half gathered by id -- so that a
    // pass moves 8-byte (key, id) pairs instead of 12-byte ones
    uint32_t* ka = reinterpret_cast<uint32_t*>(k0);  // [N] sort keys
    uint32_t* lo_by_id = ka + N;                      // [N]
    uint32_t* kb = reinterpret_cast<uint32_t*>(k1);  // [N] sort scratch
    uint32_t* hi_by_id = kb + N;                      // [N]
    LCP_TIMED_LAUNCH(k_keys_word0, blocks_for(N, 256), 256, 0, s, tk, f, N, ka, lo_by_id, hi_by_id, v0);
    uint32_t* ks;
    uint32_t* vs;
    // the low-half sort's last pass writes each row's high half as its key
    rc = radix_sort_pairs_u32(ka, v0, kb, v1, N, 32, w, s, &ks, &vs, hi_by_id);
    if (rc == LCP_OK) rc = radix_sort_pairs_u32(ka, v0, kb, v1, N, 32, w, s, &ks, &vs);
    if (rc) {
        cleanup();
        return rc;
    }
    LCP_TIMED_LAUNCH(k_ids_eq, blocks_for(N, 256), 256, 0, s, vs, ks, lo_by_id, N, ids_out, eq);
    uint32_t m = 0, G = 0;
    // Rows tied on word 0: tie groups of up to kMidMax rows are ranked directly
    // on their remaining words (found straight from eq); only groups of more
    // than kMidMax rows (if any) need the word-by-word LSD rounds below.
    uint32_t* big_start = act2;  // free until the LSD rounds
    uint32_t* big_len = idx2;
    uint32_t* cnt = w.total + 2;  // [0] listed groups, [1] rows in groups of more than kMidMax
    const unsigned fill = (unsigned)sm_count() * 8;
    auto sort_groups = [&]() -> int {
        LCP_CUDA_TRY(cudaMemsetAsync(cnt, 0, 2 * sizeof(uint32_t), s));
        LCP_TIMED_LAUNCH(k_group_scan_sort, fill, 256, 0, s, tk, f, eq, N, ids_out, big_start, big_len, cnt, cnt + 1);
        LCP_TIMED_LAUNCH(k_group_sort_mid, fill, 1024, 0, s, tk, f, ids_out, big_start, big_len, cnt, cnt + 1);
        return LCP_OK;
    };
    if (huge_host) {
        // without waiting for the device: the rows in groups of more than
        // kMidMax are counted into *huge_host, which the caller reads after its
        // final synchronise (and rebuilds exactly, here with huge_host ==
        // nullptr, if nonzero)
        if (f.W > 1) {
            rc = sort_groups();
            if (rc == LCP_OK) {
                const cudaError_t e = cudaMemcpyAsync(huge_host, cnt + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
                if (e != cudaSuccess) rc = cuda_status(e);
            }
        }
        cleanup();
        return rc;
    }
    rc = tie_compact(eq, N, act, grp, &m, &G, w, s);
    if (rc == 0 && m > 0 && f.W > 1) {
        rc = sort_groups();
        if (rc == LCP_OK) {
            cudaError_t e = cudaMemcpyAsync(w.h_total + 10, cnt + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) rc = cuda_status(e);
            else if (w.h_total[10] == 0) m = 0;  // every tie resolved
        }
    } else if (f.W == 1) {
        m = 0;  // one word: rows tied on it are equal and already in id order
    }
    // rounds 1..W-1 on the rows whose prefix is still shared
    for (int r = 1; rc == 0 && r < f.W && m > 0; ++r) {
        LCP_TIMED_LAUNCH(k_keys_active, blocks_for(m, 256), 256, 0, s, tk, f, N, ids_out, act, m, r, k0,
                   v0);
        uint64_t* ks64;
        rc = radix_sort_pairs_u64(k0, v0, k1, v1, m, 64, w, s, &ks64, &vs);
        if (rc) break;
        LCP_TIMED_LAUNCH(k_group_keys, blocks_for(m, 256), 256, 0, s, ks64, vs, grp, m, kbi, gk, gv);
        int gbits = 0;
        while (gbits < 32 && (1ull << gbits) < (uint64_t)G) ++gbits;
        uint32_t *gks, *fv;
        rc = radix_sort_pairs_u32(gk, gv, gk1, gv1, m, gbits, w, s, &gks, &fv);
        if (rc) break;
        LCP_TIMED_LAUNCH(k_apply_gather, blocks_for(m, 256), 256, 0, s, fv, ids_out, act, kbi, grp, m,
                   newid, fkey, fgrp);
        LCP_TIMED_LAUNCH(k_apply_scatter, blocks_for(m, 256), 256, 0, s, newid, act, fkey, fgrp, m,
                   ids_out, eq);
        uint32_t m2 = 0, G2 = 0;
        rc = tie_compact(eq, m, idx2, grp2, &m2, &G2, w, s);
        if (rc) break;
        if (m2) LCP_TIMED_LAUNCH(k_remap_active, blocks_for(m2, 256), 256, 0, s, act, idx2, m2, act2);
        uint32_t* t = act;
        act = act2;
        act2 = t;
        t = grp;
        grp = grp2;
        grp2 = t;
        m = m2;
        G = G2;
    }
    cleanup();
    return rc;
}

int gather_rows_and_lcp(const void* tokens, const RowFmt& f, int64_t N, const int32_t* ids,
                        lcp_buffers& b, int W, cudaStream_t s) {
    if (N <= 0) return LCP_OK;
    const bool vec = f.aligned8 && (W % 2 == 0) && (f.row_bytes % 16 == 0) &&
                     ((reinterpret_cast<uintptr_t>(tokens) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(b.rows) & 15) == 0);
    const int half = W / 2;
    if (vec && half <= 32 && (32 % half) == 0) {
        const int64_t warps = (N + (int64_t)(32 / half) * kGatherSteps - 1) / ((int64_t)(32 / half) * kGatherSteps);
        LCP_TIMED_LAUNCH(k_gather_rows_lcp, blocks_for(warps * 32, 256), 256, 0, s,
                         reinterpret_cast<const uint8_t*>(tokens), f, N, ids, b.rows, b.head, b.H);
        return LCP_OK;
    }
    if (vec) {
        LCP_TIMED_LAUNCH(k_gather_rows_v2, blocks_for(N * (W / 2), 256), 256, 0, s,
                   reinterpret_cast<const uint8_t*>(tokens), f, N, ids, b.rows, b.head);
    } else {
        LCP_TIMED_LAUNCH(k_gather_rows, blocks_for(N * W, 256), 256, 0, s,
                   reinterpret_cast<const uint8_t*>(tokens), f, N, ids, b.rows, b.head);
    }
    return adjacent_lcp(b.rows, N, W, f.L, f.tpw, f.bits, b.H, s);
}

int adjacent_lcp(const uint64_t* rows, int64_t N, int W, int L, int tpw, int bits, uint8_t* H,
                 cudaStream_t s) {
    if (N <= 0) return LCP_OK;
    LCP_TIMED_LAUNCH(k_adjacent_lcp, blocks_for(N, 256), 256, 0, s, rows, N, W, L, tpw, bits, H);
    return LCP_OK;
}

SideStream* side_stream() {
    static thread_local SideStream ss[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    SideStream& x = ss[dev];
    if (!x.s2) {
        if (cudaStreamCreateWithFlags(&x.s2, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&x.s3, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&x.fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&x.join, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&x.fork3, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&x.join3, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            x = SideStream();
            return nullptr;
        }
    }
    return &x;
}

// Sparse table of the K smallest ids over runs of 2^j blocks (reads the
// sorted blocks).
static int build_sparse_table(lcp_index_s* x, int64_t nblk, cudaStream_t s) {
    const int K = x->K;
    const int64_t lstride = x->nblk_cap * K;
    const int E = K / 32;
    if (K % 32 == 0 && (E == 1 || E == 2 || E == 4)) {  // K = 96 takes the shared-memory merge below
        const int G = E == 1 ? StRegsShape<1>::G : (E == 2 ? StRegsShape<2>::G : StRegsShape<4>::G);
        const int P = E == 1 ? StRegsShape<1>::P : (E == 2 ? StRegsShape<2>::P : StRegsShape<4>::P);
        for (int j = 1; j <= x->st_levels_cap && (1ll << j) <= nblk;) {
            int g = 1;
            while (g < G && j + g <= x->st_levels_cap && (1ll << (j + g)) <= nblk) ++g;
            const int64_t half = 1ll << (j - 1);
            StValid vb = {};
            for (int r = 0; r < g; ++r) vb.v[r] = nblk - (1ll << (j + r)) + 1;
            const int64_t prev_valid = nblk - half + 1;  // level j-1 (level 0: the blocks)
            const uint32_t* prev = j == 1 ? x->sblk : x->st + (int64_t)(j - 2) * lstride;
            const int64_t pstride = j == 1 ? kBlk : K;
            uint32_t* out = x->st + (int64_t)(j - 1) * lstride;
            const unsigned grid = blocks_for((vb.v[0] + P - 1) / P * 32, 256);
            if (E == 1)
                LCP_TIMED_LAUNCH((k_st_levels_regs<1, StRegsShape<1>::G, StRegsShape<1>::P>), grid, 256, 0, s, prev,
                                 pstride, prev_valid, half, g, lstride, vb, out);
            else if (E == 2)
                LCP_TIMED_LAUNCH((k_st_levels_regs<2, StRegsShape<2>::G, StRegsShape<2>::P>), grid, 256, 0, s, prev,
                                 pstride, prev_valid, half, g, lstride, vb, out);
            else
                LCP_TIMED_LAUNCH((k_st_levels_regs<4, StRegsShape<4>::G, StRegsShape<4>::P>), grid, 256, 0, s, prev,
                                 pstride, prev_valid, half, g, lstride, vb, out);
            j += g;
        }
        return LCP_OK;
    }
    // g levels per launch (recomputation grows as 2^g, so g shrinks as K grows)
    const int gmax = K <= 32 ? kStMaxGroup : (K <= 64 ? 2 : 1);
    for (int j = 1; j <= x->st_levels_cap && (1ll << j) <= nblk;) {
        int g = 1;
        while (g < gmax && j + g <= x->st_levels_cap && (1ll << (j + g)) <= nblk) ++g;
        const int64_t half = 1ll << (j - 1);
        int64_t valid[3] = {0, 0, 0};
        for (int r = 0; r < g; ++r) valid[r] = nblk - (1ll << (j + r)) + 1;
        const uint32_t* prev = j == 1 ? x->sblk : x->st + (int64_t)(j - 2) * lstride;
        const int64_t pstride = j == 1 ? kBlk : K;
        uint32_t* out = x->st + (int64_t)(j - 1) * lstride;
        LCP_TIMED_LAUNCH(k_st_levels, blocks_for(valid[0] * 32, 256), 256, (size_t)8 * (g > 1 ? 6 : 3) * K * sizeof(uint32_t), s,
                   prev, pstride, half, g, K, lstride, valid[0], valid[1], valid[2], out);
        j += g;
    }
    return LCP_OK;
}

// Two branches after the rows, ids, head and H exist:
//   side: pos and the buckets, then (after the sorted blocks) the sparse table
//   main: the min tree and sorted blocks, then the heavy trie nodes
// joined before the nodes' lists, which read the sparse table, pos and the
// buckets.
int build_aux(lcp_index_s* x, cudaStream_t s, bool merged) {
    const int64_t N = x->N;
    lcp_buffers& b = x->buf[x->cur];
    if (N <= 0) return LCP_OK;
    SideStream* ss = side_stream();
    cudaStream_t s2 = ss ? ss->s2 : s;  // without a side stream, one stream
    auto fork = [&]() -> cudaError_t {
        if (s2 == s) return cudaSuccess;
        cudaError_t e = cudaEventRecord(ss->fork, s);
        return e == cudaSuccess ? cudaStreamWaitEvent(s2, ss->fork, 0) : e;
    };
    LCP_CUDA_TRY(fork());
    if (!merged) {  // an insert's merge pass already wrote pos and the buckets
        LCP_TIMED_LAUNCH(k_inverse, blocks_for(N, 256), 256, 0, s2, b.ids, N, x->pos);
        LCP_TIMED_LAUNCH(k_buckets, blocks_for((1ll << x->bits) + 1, 256), 256, 0, s2, b.head, N, x->bits, x->bkt);
    }
    // depth-2 tables of the largest depth-1 buckets, on a third branch (only
    // the search reads them): joined at the end
    cudaStream_t s3 = ss && s2 != s ? ss->s3 : s2;
    const bool sub3 = x->sub_idx && !merged;
    if (sub3) {
        if (s3 != s2) {
            LCP_CUDA_TRY(cudaEventRecord(ss->fork3, s2));
            LCP_CUDA_TRY(cudaStreamWaitEvent(s3, ss->fork3, 0));
        }
        LCP_CUDA_TRY(cudaMemsetAsync(x->sub_count, 0, sizeof(uint32_t), s3));
        LCP_TIMED_LAUNCH(k_sub_assign, blocks_for(1ll << x->bits, 256), 256, 0, s3, x->bkt, x->bits, x->sub_idx,
                         x->sub_count);
        LCP_TIMED_LAUNCH(k_sub_mark, blocks_for(N, 256), 256, 0, s3, b.head, N, x->bits, x->sub_idx, x->sub);
    }
    {
        const int T = (int)(N < kTopLevels ? N : kTopLevels);
        LCP_TIMED_LAUNCH(k_top_sample, blocks_for(T, 256), 256, 0, s2, b.head, N, T, x->top);
    }
    // min tree over H: level j+1 = minima of 32 consecutive level-j entries,
    // built while a level has more than 32 entries
    int64_t len = N;
    x->hlen[0] = N;
    int lev = 0;
    int64_t off = 0;
    while (len > 32 && lev < kMaxHLev) {
        const int64_t nl = (len + 31) / 32;
        ++lev;
        x->hoff[lev] = off;
        x->hlen[lev] = nl;
        off += nl;
        len = nl;
    }
    x->hlev = lev;
    // levels 1..3 of the tree and the sorted blocks in one launch
    const int64_t nblk = (N + kBlk - 1) / kBlk;
    AuxArgs a;
    a.H = b.H;
    a.N = N;
    a.hmin = x->hmin;
    a.lev = lev < 3 ? lev : 3;
    for (int j = 1; j <= 3; ++j) {
        a.hoff[j - 1] = x->hoff[j];
        a.hlen[j - 1] = j <= lev ? x->hlen[j] : 0;
    }
    a.tree_ctas = lev > 0 ? blocks_for(N, kTreeChunk) : 0;
    a.ids = b.ids;
    a.nblk = nblk;
    a.sblk = x->sblk;
    a.soff = x->soff;
    LCP_TIMED_LAUNCH(k_aux_tree_blocks, a.tree_ctas + blocks_for(nblk, kAuxThreads / 32), kAuxThreads, 0, s, a);
    LCP_CUDA_TRY(fork());
    int rc = build_sparse_table(x, nblk, s2);
    for (int j = 4; j <= lev; ++j)  // only past 2^20 rows
        LCP_TIMED_LAUNCH(k_min32, blocks_for(x->hlen[j], 256), 256, 0, s, x->hmin + x->hoff[j - 1], x->hlen[j - 1],
                   x->hmin + x->hoff[j], x->hlen[j]);
    if (rc == LCP_OK) rc = build_tie_lists_nodes(x, s);
    if (s2 != s) {  // join (also on an error, so that a capture stays well-formed)
        LCP_CUDA_TRY(cudaEventRecord(ss->join, s2));
        LCP_CUDA_TRY(cudaStreamWaitEvent(s, ss->join, 0));
    }
    if (rc == LCP_OK) rc = build_tie_lists_fill(x, s);
    if (sub3 && s3 != s2) {  // join the third branch (also on an error)
        LCP_CUDA_TRY(cudaEventRecord(ss->join3, s3));
        LCP_CUDA_TRY(cudaStreamWaitEvent(s, ss->join3, 0));
    }
    return rc;
}

DevIndex dev_view(const lcp_index_s* x) {
    DevIndex d;
    const lcp_buffers& b = x->buf[x->cur];
    d.N = x->N;
    d.W = x->W;
    d.L = x->L;
    d.tpw = x->tpw;
    d.bits = x->bits;
    d.K = x->K;
    d.nblk = (x->N + kBlk - 1) / kBlk;
    d.hlev = x->hlev;
    int st = 0;
    while (st < x->st_levels_cap && (1ll << (st + 1)) <= d.nblk) ++st;
    d.st_levels = st;
    d.rows = b.rows;
    d.head = b.head;
    d.ids = b.ids;
    d.H = b.H;
    d.pos = x->pos;
    d.hmin = x->hmin;
    for (int i = 0; i <= kMaxHLev; ++i) {
        d.hoff[i] = x->hoff[i];
        d.hlen[i] = x->hlen[i];
    }
    d.hlen[0] = x->N;
    d.sblk = x->sblk;
    d.soff = x->soff;
    d.st = x->st;
    d.st_stride = x->nblk_cap;
    d.bkt = x->bkt;
    d.sub_idx = x->sub_idx;
    d.sub = x->sub;
    d.top = x->top;
    d.top_n = (int)(x->N < kTopLevels ? x->N : kTopLevels);
    d.tbl = x->tbl;
    d.tlists = x->tlists;
    d.tlpos = x->tlpos;
    d.bkt_list = x->bkt_list;
    d.L1 = x->L + 1;
    d.status = x->status;
    return d;
}

}  // namespace lcph
