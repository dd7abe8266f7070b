// Full scan top-k: LCP of every query against all N rows (the paper's "full
// scan" baseline, Sec. 7), no index.
//
//   k_pack_plane0   word 0 of every row, packed, into one contiguous plane
//                   (8 bytes a row: 16 MB at N=2M, so it stays in L2 while
//                   thousands of query tiles stream over it).
//   k_scan_partial  grid = (query tiles) x (N slices); a thread owns one query
//                   and the k best keys (255-LCP)<<32 | id of its slice.
//                   Rows arrive in increasing id, so once k rows are held a
//                   row matters only with an LCP above a level `worst` that
//                   k held rows reach; that test (the first worst+1 tokens
//                   equal) is one compare of word 0's XOR with q against a
//                   power of two, screened eight rows at a time on the
//                   words' upper halves (two 16-byte shared-memory loads, a
//                   range test per row as a multiply-add on the FMA pipe and
//                   a minimum on the ALU pipe), and only rows passing it pay
//                   for an exact LCP over the remaining words.  Rows taken are
//                   appended to a log in id order; when the log holds
//                   k + kLogSlack rows, worst is raised to the k-th largest
//                   LCP and the log cut back to k rows (those above worst
//                   and the earliest at it) -- a few passes over the log
//                   every kLogSlack rows instead of a heap sift per row.
//   k_scan_merge    keys are unique, so the k smallest over a query's slice
//                   lists are order independent: sort G lists' keys in shared
//                   memory, keep k, repeat until one list is left, write out.
#include "scan.cuh"

namespace lcpk {

constexpr int kScanTile = 2048;     // plane-0 words staged per smem tile
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
                              uint64_t* __restrict__ plane0) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) plane0[i] = row_word0(row_of(tokens, i, f), f);
}

// Word-0 mask that tests "the first t tokens are equal" (t <= tpw).
__device__ __forceinline__ uint64_t prefix_mask(int t, int bits) {
    int b = t * bits;
    return b >= 64 ? ~0ull : (b == 0 ? 0ull : (~0ull << (64 - b)));
}

__global__ void __launch_bounds__(kScanPartialThreads) k_scan_partial(const uint8_t* __restrict__ tokens,
                                                      const uint64_t* __restrict__ plane0, RowFmt f,
                                                      int64_t N, const uint8_t* __restrict__ queries,
                                                      RowFmt qf, int64_t Q, int k, int cap, int64_t slice,
                                                      uint64_t* __restrict__ lists) {
    __shared__ __align__(16) uint64_t tile[kScanTile];
    __shared__ __align__(16) uint32_t tile_hi[kScanTile];  // the words' upper halves
    const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t s0 = (int64_t)blockIdx.y * slice;
    const int64_t s1 = s0 + slice < N ? s0 + slice : N;
    const bool active = qi < Q;
    const uint8_t* qrow = active ? row_of(queries, qi, qf) : nullptr;
    const uint64_t q0 = active ? pack_word(qrow, 0, qf) : 0;
    // the thread's log: keys (255 - LCP) << 32 | id of the rows taken, in id
    // order (rows arrive in increasing id), at most cap of them
    uint64_t* log = lists + ((int64_t)blockIdx.y * Q + (active ? qi : 0)) * cap;
    int n = 0;
    int worst = -1;  // -1 until k rows are logged; then a level with >= k logged rows at or above it
    // A row can matter only with LCP > worst: its first worst + 1 tokens
    // equal to q's, i.e. (r ^ q0) < T for T = 2^(64 - (worst + 1) * bits)
    // (T = 1 past word 0: word 0 all equal).  The screen on the upper halves:
    // (r ^ q0) < T implies (r_hi ^ q_hi) < max(T >> 32, 1), the two tests
    // being equal when T >= 2^32 (the tokens to match lie in the upper half).
    uint64_t T = 0;
    uint32_t Th = 0;
    const uint32_t qh = (uint32_t)(q0 >> 32);
    // The screen as a range test: (r_hi ^ q_hi) < Th = 2^m iff
    // r_hi - lo < Th (mod 2^32) with lo = q_hi rounded down to a multiple of
    // 2^m.  The subtraction is written as a multiply-add by a factor the
    // compiler cannot fold (1 for every legal block size, <= 128 threads),
    // so that it runs on the FMA pipe beside the minimums on the ALU pipe.
    uint32_t neg_lo = 0;
    const uint32_t unit = (blockDim.x + 127u) / 128u;
    auto sub_lo = [&](uint32_t x) {
        uint32_t d;
        asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(x), "r"(unit), "r"(neg_lo));
        return d;
    };
    auto lam_of = [](uint64_t e) { return 255 - (int)(e >> 32); };
    // Raises worst to the largest w with >= k logged rows of LCP >= w and
    // keeps the rows above w and the earliest (smallest-id) ones at w, k in
    // all.  A row dropped here, or refused later for LCP <= worst, has k
    // logged rows of smaller id and no smaller LCP: it is in no top k.
    auto compact = [&]() {
        int w, above;
        if (worst < 0) {  // the first k rows: w = their smallest LCP, all kept
            w = 255;
            for (int i = 0; i < n; ++i) w = min(w, lam_of(log[i]));
            above = 0;
            for (int i = 0; i < n; ++i) above += lam_of(log[i]) > w;
        } else {
            w = worst;
            for (;;) {
                int c = 0;
                for (int i = 0; i < n; ++i) c += lam_of(log[i]) > w;
                if (c < k) {
                    above = c;
                    break;
                }
                ++w;
            }
        }
        int eq = k - above;
        int m = 0;
        for (int i = 0; i < n; ++i) {
            const uint64_t e = log[i];
            const int l = lam_of(e);
            if (l > w || (l == w && eq-- > 0)) log[m++] = e;
        }
        n = m;
        worst = w;
        const int b = (worst + 1) * f.bits;
        T = b >= 64 ? 1ull : (1ull << (64 - b));
        Th = b >= 32 ? 1u : (uint32_t)(T >> 32);
        neg_lo = 0u - (qh & ~(Th - 1u));
    };
    auto row_at = [&](int64_t id, uint64_t r) {  // a row that may matter
        int lam;
        const uint64_t x = r ^ q0;
        if (x) {
            lam = __clzll((long long)x) / f.bits;
        } else {
            lam = f.L;
            const uint8_t* row = row_of(tokens, id, f);
            for (int w = 1; w < f.W; ++w) {
                const uint64_t y = pack_word(row, w, f) ^ pack_word(qrow, w, qf);
                if (y) {
                    lam = w * f.tpw + (__clzll((long long)y) / f.bits);
                    break;
                }
            }
        }
        if (lam > f.L) lam = f.L;
        if (worst >= 0 && lam <= worst) return;
        log[n++] = ((uint64_t)(255 - lam) << 32) | (uint64_t)id;
        if (worst < 0 ? n == k : n == cap) compact();
    };
    for (int64_t t0 = s0; t0 < s1; t0 += kScanTile) {
        const int tn = (int)(s1 - t0 < kScanTile ? s1 - t0 : kScanTile);
        __syncthreads();
        for (int j = threadIdx.x; j < tn; j += blockDim.x) {
            const uint64_t w = plane0[t0 + j];
            tile[j] = w;
            tile_hi[j] = (uint32_t)(w >> 32);
        }
        __syncthreads();
        if (!active) continue;
        int j = 0;
        // the first k rows are logged unconditionally (the same rows for
        // every thread of the CTA: all start at s0)
        for (; j < tn && worst < 0; ++j) row_at(t0 + j, tile[j]);
        for (; j < tn && (j & 7); ++j)
            if ((tile[j] ^ q0) < T) row_at(t0 + j, tile[j]);
        // eight rows per step: two 16-byte loads of upper halves, their XORs
        // with q's and a minimum; rows pass rarely
        for (; j + 8 <= tn; j += 8) {
            const uint4 a = *reinterpret_cast<const uint4*>(tile_hi + j);
            const uint4 b = *reinterpret_cast<const uint4*>(tile_hi + j + 4);
            const uint32_t m = min(min(min(sub_lo(a.x), sub_lo(a.y)), min(sub_lo(a.z), sub_lo(a.w))),
                                   min(min(sub_lo(b.x), sub_lo(b.y)), min(sub_lo(b.z), sub_lo(b.w))));
            if (m >= Th) continue;
#pragma unroll 1
            for (int u = 0; u < 8; ++u) {
                const uint64_t r = tile[j + u];
                if ((r ^ q0) < T) row_at(t0 + j + u, r);
            }
        }
        for (; j < tn; ++j)
            if ((tile[j] ^ q0) < T) row_at(t0 + j, tile[j]);
    }
    if (active) {
        if (n > k) compact();
        for (int j = n; j < k; ++j) log[j] = kKeyInf;
    }
}

// Reduces groups of G lists of k keys per query to one list each (sorted when
// `final`, which then writes ids and LCPs); list l of query q starts at
// in[(l * Q + q) * in_stride].  grid = (Q, groups).
__global__ void __launch_bounds__(256) k_scan_merge(const uint64_t* __restrict__ in, int in_stride,
                                                    int64_t Q, int k, int nlists, int G, int P,
                                                    uint64_t* __restrict__ out, int final_pass,
                                                    int32_t* __restrict__ out_ids,
                                                    uint8_t* __restrict__ out_lcp) {
    extern __shared__ uint64_t keys[];
    const int64_t q = blockIdx.x;
    const int g = blockIdx.y;
    const int l0 = g * G;
    const int nl = nlists - l0 < G ? nlists - l0 : G;
    const int n = nl * k;
    for (int t = threadIdx.x; t < P; t += blockDim.x) {
        uint64_t v = kKeyInf;
        if (t < n) {
            int l = t / k, j = t - l * k;
            v = in[((int64_t)(l0 + l) * Q + q) * in_stride + j];
        }
        keys[t] = v;
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < P; t += blockDim.x) {
                int u = t ^ stride;
                if (u > t) {
                    uint64_t a = keys[t], b = keys[u];
                    bool up = (t & size) == 0;
                    if ((a > b) == up) {
                        keys[t] = b;
                        keys[u] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    if (final_pass) {
        for (int j = threadIdx.x; j < k; j += blockDim.x) {
            uint64_t v = keys[j];
            out_ids[q * k + j] = v == kKeyInf ? -1 : (int32_t)(uint32_t)v;
            out_lcp[q * k + j] = v == kKeyInf ? 0 : (uint8_t)(255 - (int)(v >> 32));
        }
    } else {
        for (int j = threadIdx.x; j < k; j += blockDim.x) out[((int64_t)g * Q + q) * k + j] = keys[j];
    }
}


// ---- small batches: threshold selection ----
//
// With few queries the per-thread heaps above leave most of the GPU idle (one
// thread per query and slice) and their merge dominates.  Such batches take
// the answer from the LCP distribution instead: d* is the largest d with at
// least k rows of LCP >= d (0 when N < k); every row with LCP > d* is in the
// answer (nA < k of them), and the other kp = min(k - nA, #LCP-d* rows) slots
// go to the rows of LCP exactly d* in ascending id order.
//   k_sel_count    a warp per (query, slice of ids): rows with LCP >= d for
//                  d = 1..L, per slice and (one atomic per CTA) in total; the
//                  exact LCP is computed only for rows whose first token
//                  matches the query's;
//   k_sel_pick     a CTA per query: d*, nA, kp and, per slice, the LCP-d*
//                  rows in the slices before it;
//   k_sel_collect  a warp per (query, slice) walks only slices that hold
//                  answer rows, and stops once it has found them: LCP > d*
//                  into unordered slots, LCP-d* rows at their rank; the
//                  query's last CTA to finish sorts the nA keys and writes
//                  A, the tie rows, then padding.

constexpr int kSelWarps = 8;
constexpr int kSelBins = 16;
constexpr int kSelMaxS = 8192;  // slices per query at most  // LCPs below this are counted per lane, larger ones by shared atomics
constexpr int kMaxScanW = (LCP_MAX_L + 3) / 4;  // packed words of the longest uint16 row

struct SelArgs {
    const uint8_t* tokens;
    const uint64_t* plane0;  // packed word 0 of every row, or null: read from the tokens
    RowFmt f;
    int64_t N;
    const uint8_t* queries;
    RowFmt qf;
    int64_t Q;
    int k;
    int S;              // slices per query
    int64_t slice;      // rows per slice (the last may be shorter)
    uint32_t* ge;       // [Q][L][S]: rows of slice s with LCP >= d, d = 1..L (zeroed first)
    uint32_t* tot;      // [Q][L]: the same over all rows (zeroed before k_sel_count)
    int32_t* meta;      // [Q][8]: d*, nA, kp, the A slot counter, the collect pass's CTA ticket
    uint32_t* tie_lo;   // [Q][S]: LCP-d* rows in the slices before this one
    uint64_t* abuf;     // [Q][k]: keys (255 - LCP) << 32 | id of the rows with LCP > d*
    int32_t* tbuf;      // [Q][k]: ids of the first kp rows of LCP d*
};

__device__ __forceinline__ uint64_t sel_word0(const SelArgs& a, int64_t t) {
    return a.plane0 ? a.plane0[t] : row_word0(row_of(a.tokens, t, a.f), a.f);
}

// Exact LCP of row t with the query, given x = word0(t) ^ q0 (qw: the
// query's packed words).
__device__ __forceinline__ int sel_lcp(const SelArgs& a, int64_t t, uint64_t x, const uint64_t* qw) {
    const RowFmt& f = a.f;
    if (x) return lcp_at(0, x, f);
    const uint8_t* row = row_of(a.tokens, t, f);
    if (f.aligned8) {  // four words per round trip rather than one
        const unsigned long long* rw = reinterpret_cast<const unsigned long long*>(row);
        for (int w0 = 1; w0 < f.W; w0 += 4) {
            uint64_t v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) v[j] = w0 + j < f.W ? __ldg(rw + w0 + j) : 0ull;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint64_t y = w0 + j < f.W ? msb_first(v[j], f.tb) ^ qw[w0 + j] : 0ull;
                if (y) return lcp_at(w0 + j, y, f);
            }
        }
        return f.L;
    }
    for (int w = 1; w < f.W; ++w) {
        const uint64_t y = pack_word(row, w, f) ^ qw[w];
        if (y) return lcp_at(w, y, f);
    }
    return f.L;
}

__device__ __forceinline__ void sel_slice(const SelArgs& a, int s, int64_t* s0, int64_t* s1) {
    *s0 = (int64_t)s * a.slice;
    const int64_t e = *s0 + a.slice;
    *s1 = e < a.N ? e : a.N;
}

__global__ void __launch_bounds__(kSelWarps * 32, 4) k_sel_count(SelArgs a) {
    __shared__ uint64_t qw[kMaxScanW];
    __shared__ uint32_t hist[kSelWarps][LCP_MAX_L + 1];
    __shared__ uint32_t lanecnt[kSelWarps][kSelBins][32];  // [l][lane]: bank = lane, no conflicts
    const int64_t q = blockIdx.y;
    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const int L = a.f.L;
    const uint8_t* qrow = row_of(a.queries, q, a.qf);
    for (int w = threadIdx.x; w < a.f.W; w += blockDim.x) qw[w] = pack_word(qrow, w, a.qf);
    uint32_t* h = hist[warp];
    uint32_t* lc = &lanecnt[warp][0][lane];
    for (int d = (int)lane; d <= L; d += 32) h[d] = 0;
#pragma unroll
    for (int d = 0; d < kSelBins; ++d) lc[d * 32] = 0;
    __syncthreads();
    const int s = blockIdx.x * kSelWarps + warp;
    if (s < a.S) {
        int64_t s0, s1;
        sel_slice(a, s, &s0, &s1);
        const uint64_t q0 = qw[0];
        const uint32_t qh = (uint32_t)(q0 >> 32);
        const uint32_t lim = 1u << (32 - a.f.bits);  // (word 0 ^ q0) >> 32 below it: first token agrees
        // 128 rows per step; the next step's words are loaded before this
        // step's are tested
        uint64_t r[4], nx[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t t = s0 + u * 32 + lane;
            r[u] = t < s1 ? sel_word0(a, t) : ~q0;
        }
        for (int64_t b = s0; b < s1; b += 128) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t t = b + 128 + u * 32 + lane;
                nx[u] = t < s1 ? sel_word0(a, t) : ~q0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool hit = ((uint32_t)(r[u] >> 32) ^ qh) < lim;
                if (!__any_sync(0xffffffffu, hit)) continue;
                if (hit) {
                    const int l = sel_lcp(a, b + u * 32 + lane, r[u] ^ q0, qw);  // >= 1
                    if (l < kSelBins) lc[l * 32] += 1;
                    else atomicAdd(h + l, 1u);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) r[u] = nx[u];
        }
        __syncwarp();
        for (int d = 1; d < kSelBins && d <= L; ++d) {
            const uint32_t v = __reduce_add_sync(0xffffffffu, lc[d * 32]);
            if (lane == 0) h[d] += v;
        }
        __syncwarp();
        // suffix sums (rows with LCP >= d), from d = L down to 1, stored per
        // slice where nonzero and kept in h for the CTA's total
        uint32_t* out = a.ge + (size_t)q * L * a.S + s;
        uint32_t carry = 0;
        for (int c = ((L - 1) / 32) * 32 + 1; c >= 1; c -= 32) {
            const int d = c + (int)lane;
            uint32_t v = d <= L ? h[d] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_down_sync(0xffffffffu, v, o);
                if ((int)lane + o < 32) v += y;
            }
            v += carry;
            __syncwarp();
            if (d <= L) {
                if (v) out[(size_t)(d - 1) * a.S] = v;
                h[d] = v;
            }
            carry = __shfl_sync(0xffffffffu, v, 0);
        }
    }
    __syncthreads();
    for (int d = threadIdx.x + 1; d <= L; d += blockDim.x) {
        uint32_t v = 0;
#pragma unroll
        for (int w = 0; w < kSelWarps; ++w) v += hist[w][d];
        if (v) atomicAdd(a.tot + (size_t)q * L + (d - 1), v);
    }
}

__global__ void __launch_bounds__(1024) k_sel_pick(SelArgs a) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t tie[kSelMaxS];  // LCP-d* rows per slice, then their exclusive prefix
    const int64_t q = blockIdx.x;
    const int L = a.f.L, S = a.S;
    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t* tot = a.tot + (size_t)q * L;
    // the counts fall with d, so d* is the number of d in 1..L reaching k
    const int dstar = __syncthreads_count((int)threadIdx.x < L && tot[threadIdx.x] >= (uint32_t)a.k);
    const uint32_t nA = dstar < L ? tot[dstar] : 0u;
    const uint32_t atd = dstar == 0 ? (uint32_t)a.N : tot[dstar - 1];
    const uint32_t kp = min((uint32_t)a.k - nA, atd - nA);
    const uint32_t* g = a.ge + (size_t)q * L * S;  // level-major: these reads are contiguous
    {
        // S <= kSelMaxS = 8 x 1024: each thread's loads issued together
        uint32_t hv[kSelMaxS / 1024], lv[kSelMaxS / 1024];
#pragma unroll
        for (int i = 0; i < kSelMaxS / 1024; ++i) {
            const int s = (int)threadIdx.x + i * 1024;
            hv[i] = s < S && dstar > 0 ? g[(size_t)(dstar - 1) * S + s] : 0u;
            lv[i] = s < S && dstar < L ? g[(size_t)dstar * S + s] : 0u;
        }
#pragma unroll
        for (int i = 0; i < kSelMaxS / 1024; ++i) {
            const int s = (int)threadIdx.x + i * 1024;
            if (s >= S) break;
            int64_t s0, s1;
            sel_slice(a, s, &s0, &s1);
            tie[s] = (dstar == 0 ? (uint32_t)(s1 - s0) : hv[i]) - lv[i];
        }
    }
    __syncthreads();
    const int per = (S + (int)blockDim.x - 1) / (int)blockDim.x;
    const int sb = (int)threadIdx.x * per;
    const int se = sb + per < S ? sb + per : S;
    uint32_t sum = 0;
    for (int s = sb; s < se; ++s) sum += tie[s];
    uint32_t v = sum;  // inclusive scan over the block
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= (unsigned)o) v += y;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (int)lane < nwarps ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= (unsigned)o) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    uint32_t run = v - sum + (warp > 0 ? wsum[warp - 1] : 0u);
    for (int s = sb; s < se; ++s) {
        const uint32_t t = tie[s];
        tie[s] = run;
        run += t;
    }
    __syncthreads();
    for (int s = threadIdx.x; s < S; s += blockDim.x) a.tie_lo[(size_t)q * S + s] = tie[s];
    if (threadIdx.x == 0) {
        int32_t* m = a.meta + q * 8;
        m[0] = dstar;
        m[1] = (int32_t)nA;
        m[2] = (int32_t)kp;
        m[3] = 0;
        m[4] = 0;
    }
}

// Query q's output: the nA keys of A sorted (by a CTA, in keys[]), then the
// tie rows, then padding.
__device__ void sel_write(const SelArgs& a, int64_t q, uint64_t* keys, int32_t* __restrict__ out_ids,
                          uint8_t* __restrict__ out_lcp) {
    const int k = a.k;
    const int32_t* m = a.meta + q * 8;
    const int dstar = m[0], nA = m[1], kp = m[2];
    int P = 1;
    while (P < nA) P <<= 1;
    const uint64_t* abuf = a.abuf + q * k;
    for (int t = threadIdx.x; t < P; t += blockDim.x) keys[t] = t < nA ? abuf[t] : kKeyInf;
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
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
    const int32_t* tbuf = a.tbuf + q * k;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        int32_t id = -1;
        int l = 0;
        if (j < nA) {
            const uint64_t v = keys[j];
            id = (int32_t)(uint32_t)v;
            l = 255 - (int)(v >> 32);
        } else if (j < nA + kp) {
            id = tbuf[j - nA];
            l = dstar;
        }
        out_ids[q * k + j] = id;
        out_lcp[q * k + j] = (uint8_t)l;
    }
}

__global__ void __launch_bounds__(kSelWarps * 32) k_sel_collect(SelArgs a, int32_t* __restrict__ out_ids,
                                                                uint8_t* __restrict__ out_lcp) {
    __shared__ uint64_t qw[kMaxScanW];
    __shared__ uint64_t keys[LCP_SCAN_MAX_K];
    __shared__ int last;
    const int64_t q = blockIdx.y;
    const unsigned lane = lane_id();
    const unsigned lt = lanemask_lt();
    const int warp = threadIdx.x >> 5;
    const int L = a.f.L;
    const uint8_t* qrow = row_of(a.queries, q, a.qf);
    for (int w = threadIdx.x; w < a.f.W; w += blockDim.x) qw[w] = pack_word(qrow, w, a.qf);
    __syncthreads();
    const int s = blockIdx.x * kSelWarps + warp;
    if (s < a.S) {
        int32_t* m = a.meta + q * 8;
        const int dstar = m[0], kp = m[2];
        int64_t s0, s1;
        sel_slice(a, s, &s0, &s1);
        const uint32_t* g = a.ge + (size_t)q * L * a.S + s;
        const uint32_t atd = dstar == 0 ? (uint32_t)(s1 - s0) : g[(size_t)(dstar - 1) * a.S];
        uint32_t a_left = dstar < L ? g[(size_t)dstar * a.S] : 0u;  // rows of LCP > d* not yet met
        const uint32_t tlo = a.tie_lo[(size_t)q * a.S + s];
        const uint32_t ties_s = atd - a_left;
        const uint32_t t_need = (uint32_t)kp > tlo ? min(ties_s, (uint32_t)kp - tlo) : 0u;
        const uint64_t q0 = qw[0];
        const uint64_t first = ~0ull >> a.f.bits;
        // rows whose first min(d*, tpw) tokens match (all rows when d* = 0)
        const int dm = dstar < a.f.tpw ? dstar : a.f.tpw;
        const uint64_t mask = prefix_mask(dm, a.f.bits);
        uint64_t* abuf = a.abuf + q * a.k;
        int32_t* tbuf = a.tbuf + q * a.k;
        uint32_t seen = 0;  // LCP-d* rows of this slice met so far
        // 128 rows per step, the next step's words loaded before this step's
        // are tested (rows of a step in ascending id, as the ranks need)
        uint64_t r[4], nx[4];
    #pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t t = s0 + u * 32 + lane;
            r[u] = t < s1 ? sel_word0(a, t) : 0ull;
        }
        for (int64_t b = s0; b < s1 && (a_left > 0 || seen < t_need); b += 128) {
    #pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t t = b + 128 + u * 32 + lane;
                nx[u] = t < s1 ? sel_word0(a, t) : 0ull;
            }
    #pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (!(a_left > 0 || seen < t_need)) break;  // warp-uniform
                const int64_t t = b + u * 32 + lane;
                const bool in = t < s1;
                const uint64_t x = r[u] ^ q0;
                const bool cand = in && (x & mask) == 0;
                if (!__any_sync(0xffffffffu, cand)) continue;
                const int l = cand && x <= first ? sel_lcp(a, t, x, qw) : 0;
                const bool isA = cand && l > dstar;
                const bool isT = cand && l == dstar;
                const unsigned mA = __ballot_sync(0xffffffffu, isA);
                if (mA) {
                    uint32_t base = 0;
                    if (lane == 0) base = atomicAdd(reinterpret_cast<uint32_t*>(m + 3), (uint32_t)__popc(mA));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    const uint32_t slot = base + (uint32_t)__popc(mA & lt);
                    if (isA && slot < (uint32_t)a.k) abuf[slot] = ((uint64_t)(255 - l) << 32) | (uint64_t)t;
                    const uint32_t na = (uint32_t)__popc(mA);
                    a_left = a_left > na ? a_left - na : 0u;
                }
                const unsigned mT = __ballot_sync(0xffffffffu, isT);
                if (isT) {
                    const uint32_t rank = tlo + seen + (uint32_t)__popc(mT & lt);
                    if (rank < (uint32_t)kp) tbuf[rank] = (int32_t)t;
                }
                seen += (uint32_t)__popc(mT);
            }
    #pragma unroll
            for (int u = 0; u < 4; ++u) r[u] = nx[u];
        }
    }
    // the CTA that finishes the query's collect pass last (every CTA's
    // writes fenced before its ticket) sorts A and writes the output
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
        last = atomicAdd(reinterpret_cast<unsigned*>(a.meta + q * 8 + 4), 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    sel_write(a, q, keys, out_ids, out_lcp);
}

}  // namespace lcpk

namespace lcph {
using namespace lcpk;

// Batches up to this size take the threshold selection, larger ones the
// per-thread logs, whose screen of a row against a level k logged rows reach
// is cheaper per pair once every thread of the GPU has a query (measured on
// 2M rows of 64 uint16 tokens: the selection is 1.5x ahead at 256 queries,
// level at 512, 1.6x behind at 1,024; 3.3x ahead at 32).
constexpr int64_t kSelMaxQ = 512;

static int scan_select(const void* d_tokens, int64_t N, const RowFmt& f, const void* d_queries,
                       const RowFmt& qf, int64_t Q, int k, int32_t* d_out_ids, uint8_t* d_out_lcp,
                       cudaStream_t s) {
    const int L = f.L;
    // about 64 warps per SM over all (query, slice) pairs (two waves, so
    // that slices with long walks in the collect pass even out), whole CTAs
    // of slices, slices of >= 256 rows
    const int64_t target = (int64_t)sm_count() * 64;
    int64_t S = (target + Q - 1) / Q;
    S = (S + kSelWarps - 1) / kSelWarps * kSelWarps;
    const int64_t maxS = (N + 255) / 256;
    if (S > maxS) S = maxS;
    if (S > kSelMaxS) S = kSelMaxS;
    if (S < 1) S = 1;
    const int64_t slice = (N + S - 1) / S;
    S = (N + slice - 1) / slice;
    const bool plane = Q > 1;  // several queries re-read word 0: pack it once
    SelArgs a;
    a.tokens = reinterpret_cast<const uint8_t*>(d_tokens);
    a.plane0 = nullptr;
    a.f = f;
    a.N = N;
    a.queries = reinterpret_cast<const uint8_t*>(d_queries);
    a.qf = qf;
    a.Q = Q;
    a.k = k;
    a.S = (int)S;
    a.slice = slice;
    uint64_t* plane0 = nullptr;
    Carver cv;
    if (plane) cv.add(&plane0, (size_t)N);
    cv.add(&a.ge, (size_t)Q * S * L);
    cv.add(&a.tot, (size_t)Q * L);
    cv.add(&a.meta, (size_t)Q * 8);
    cv.add(&a.tie_lo, (size_t)Q * S);
    cv.add(&a.abuf, (size_t)Q * k);
    cv.add(&a.tbuf, (size_t)Q * k);
    void* base = nullptr;
    LCP_CUDA_TRY(cv.alloc(&base, s));
    a.plane0 = plane0;
    // the per-slice counts and the totals are adjacent: one memset zeroes both
    cudaError_t e = cudaMemsetAsync(a.ge, 0, (size_t)((char*)(a.tot + (size_t)Q * L) - (char*)a.ge), s);
    if (e != cudaSuccess) {
        cudaFreeAsync(base, s);
        return cuda_status(e);
    }
    if (plane)
        LCP_TIMED_LAUNCH(k_pack_plane0, (unsigned)((N + 255) / 256), 256, 0, s, a.tokens, f, N, plane0);
    const dim3 grid((unsigned)((S + kSelWarps - 1) / kSelWarps), (unsigned)Q);
    LCP_TIMED_LAUNCH(k_sel_count, grid, kSelWarps * 32, 0, s, a);
    LCP_TIMED_LAUNCH(k_sel_pick, (unsigned)Q, 1024, 0, s, a);
    LCP_TIMED_LAUNCH(k_sel_collect, grid, kSelWarps * 32, 0, s, a, d_out_ids, d_out_lcp);
    e = cudaFreeAsync(base, s);
    return e == cudaSuccess ? LCP_OK : cuda_status(e);
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
    const int threads = kScanPartialThreads;
    const int64_t qtiles = (Q + threads - 1) / threads;
    const int64_t target = 148 * 8;
    int64_t S = (target + qtiles - 1) / qtiles;
    int64_t maxS = (N + 1023) / 1024;
    if (S > maxS) S = maxS;
    if (S > 65535) S = 65535;
    if (S < 1) S = 1;
    int64_t slice = (N + S - 1) / S;
    S = (N + slice - 1) / slice;
    const int cap = k + kLogSlack;  // log entries per (slice, query)
    uint64_t* plane0 = nullptr;
    uint64_t* heaps = nullptr;
    LCP_CUDA_TRY(cudaMallocAsync((void**)&plane0, sizeof(uint64_t) * N, s));
    LCP_CUDA_TRY(cudaMallocAsync((void**)&heaps, sizeof(uint64_t) * (size_t)S * Q * cap, s));
    LCP_TIMED_LAUNCH(k_pack_plane0, (unsigned)((N + 255) / 256), 256, 0, s,
               reinterpret_cast<const uint8_t*>(d_tokens), f, N, plane0);
    dim3 grid((unsigned)qtiles, (unsigned)S);
    LCP_TIMED_LAUNCH(k_scan_partial, grid, threads, 0, s, reinterpret_cast<const uint8_t*>(d_tokens),
               plane0, f, N, reinterpret_cast<const uint8_t*>(d_queries), qf, Q, k, cap, slice, heaps);
    // merge: groups of G lists until one remains
    int kp2 = 1;
    while (kp2 < k) kp2 <<= 1;
    int G = kMergeCap / kp2;
    if (G < 1) G = 1;
    int64_t nl = S;
    uint64_t* cur = heaps;
    int rc = LCP_OK;
    for (;;) {
        int g = (int)(nl < G ? nl : G);
        int64_t groups = (nl + g - 1) / g;
        int P = 1;
        while (P < g * k) P <<= 1;
        size_t smem = sizeof(uint64_t) * P;
        cudaError_t e = cudaFuncSetAttribute(k_scan_merge, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(sizeof(uint64_t) * kMergeCap * 2));
        if (e != cudaSuccess) {
            rc = cuda_status(e);
            break;
        }
        bool final_pass = groups == 1;
        uint64_t* out = nullptr;
        if (!final_pass) {
            e = cudaMallocAsync((void**)&out, sizeof(uint64_t) * (size_t)groups * Q * k, s);
            if (e != cudaSuccess) {
                rc = cuda_status(e);
                break;
            }
        }
        dim3 mg((unsigned)Q, (unsigned)groups);
        LCP_TIMED_LAUNCH(k_scan_merge, mg, 256, smem, s, cur, cur == heaps ? cap : k, Q, k, (int)nl, g, P,
                   out, final_pass ? 1 : 0, d_out_ids, d_out_lcp);
        if (cur != heaps) cudaFreeAsync(cur, s);
        if (final_pass) break;
        cur = out;
        nl = groups;
    }
    cudaFreeAsync(plane0, s);
    cudaFreeAsync(heaps, s);
    return rc;
}

}  // namespace lcph
