// LSD radix sort (8-bit digits) for the index build.
//
// Each pass is reduce-then-scan: per-tile digit counts (warp-aggregated, so
// that the heavily skewed digits of Zipf-distributed tokens do not serialise
// on shared memory), then a kernel that derives each digit's base and its
// offset for the tile, ranks its tile stably (warp multisplit), stages it in
// shared memory by digit and writes it out in coalesced runs.  Up to 4,096
// tiles the count kernel also adds each tile's counts into its superblock of
// 32 tiles, and the scatter CTA sums the superblocks before its own and the
// tiles before it in its superblock (64 loads a thread, all in flight at
// once); a larger sort runs one exclusive scan per digit over the tiles
// between the two.  Either way the digit totals show a constant digit,
// whose scatter is then skipped on the device.  No CTA waits for another: a
// chained scan with look-back serialises the first wave of tiles that start
// together, and a sort pass has only one or two waves.
#include "sort.cuh"

namespace lcpk {

using lcph::kSortItems;
using lcph::kSortThreads;
using lcph::kSortTile;
using lcph::kSortSup;
constexpr int kSortWarps = kSortThreads / 32;

// Lanes of the warp whose 8-bit digit equals this lane's (invalid lanes are
// never peers).  Eight ballots: much cheaper than __match_any_sync.
__device__ __forceinline__ unsigned digit_peers(uint32_t d, bool valid) {
    unsigned peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const bool bit = (d >> b) & 1u;
        const unsigned m = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? m : ~m;
    }
    return valid ? peers : 0u;
}

// Exclusive scan of a 256-entry table by 256 threads.
__device__ __forceinline__ uint32_t block_excl_scan_256(uint32_t v, uint32_t* tmp /*8*/) {
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    uint32_t add = 0;
    for (unsigned w = 0; w < warp; ++w) add += tmp[w];
    __syncthreads();
    return add + x - v;
}

// Moves the result into buffer 0 when an odd number of passes ran, and
// maps its keys through key_of_value when the last pass (which maps them
// as it writes) was skipped.
template <typename K>
__global__ void k_result_to_buf0(const uint32_t* __restrict__ sel, int passes, const K* __restrict__ k1,
                                 const uint32_t* __restrict__ v1, K* __restrict__ k0,
                                 uint32_t* __restrict__ v0, uint32_t n,
                                 const uint32_t* __restrict__ key_of_value) {
    const bool in1 = sel[passes] != 0;
    const bool map = key_of_value != nullptr && sel[passes] == sel[passes - 1];
    if (!in1 && !map) return;
    const K* ks = in1 ? k1 : k0;
    const uint32_t* vs = in1 ? v1 : v0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t v = vs[i];
        k0[i] = map ? (K)(v < n ? key_of_value[v] : 0u) : ks[i];
        v0[i] = v;
    }
}

// Per-tile digit counts of pass `pass`: counts[d * tiles + tile].
template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_tile_counts(const K* kb0, const K* kb1, uint32_t n,
                                                              int pass, const uint32_t* __restrict__ skip,
                                                              const uint32_t* __restrict__ sel,
                                                              uint32_t* __restrict__ counts, uint32_t tiles,
                                                              uint32_t* __restrict__ sup, uint32_t sups) {
    __shared__ uint32_t wh[kSortWarps][256];
    const K* __restrict__ kin = sel[pass] ? kb1 : kb0;
    const int tid = threadIdx.x;
    const unsigned lane = lane_id();
    const int warp = tid >> 5;
    for (int i = tid; i < kSortWarps * 256; i += kSortThreads) (&wh[0][0])[i] = 0;
    const uint32_t tile = blockIdx.x;
    const uint32_t base = tile * (uint32_t)kSortTile;
    const uint32_t tile_n = min((uint32_t)kSortTile, n - base);
    const int shift = 8 * pass;
    K kk[kSortItems];
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const uint32_t idx = (uint32_t)warp * (32 * kSortItems) + (uint32_t)i * 32 + lane;
        kk[i] = idx < tile_n ? kin[base + idx] : (K)0;
    }
    __syncthreads();  // zeroed counters visible
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const uint32_t idx = (uint32_t)warp * (32 * kSortItems) + (uint32_t)i * 32 + lane;
        const bool valid = idx < tile_n;
        const uint32_t d = (uint32_t)(kk[i] >> shift) & 255u;
        const unsigned peers = digit_peers(d, valid);
        if (valid && lane == (unsigned)(__ffs(peers) - 1)) wh[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    uint32_t t = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) t += wh[w][tid];
    if (sup == nullptr) {
        counts[(size_t)tid * tiles + tile] = t;  // digit-major, for the tile scan
    } else {
        // tile-major (a warp's loads of one tile's counts are one line) and
        // added into its superblock's sums
        counts[(size_t)tile * 256 + tid] = t;
        if (t != 0) atomicAdd(sup + ((size_t)pass * sups + tile / kSortSup) * 256 + tid, t);
    }
}

// Exclusive scan of each digit's counts over the tiles (one CTA per digit);
// the digit's total goes to totals[pass][d], and a digit holding all n keys
// marks the pass as skipped (its scatter would move nothing).
__global__ void __launch_bounds__(1024) k_tile_scan(int pass, uint32_t* __restrict__ skip,
                                                    uint32_t* __restrict__ counts, uint32_t tiles,
                                                    uint32_t* __restrict__ totals, uint32_t n) {
    __shared__ uint32_t tmp[32];
    __shared__ uint32_t carry;
    const int d = blockIdx.x;
    uint32_t* col = counts + (size_t)d * tiles;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t b0 = 0; b0 < tiles; b0 += 1024) {
        const uint32_t i = b0 + threadIdx.x;
        const uint32_t v = i < tiles ? col[i] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane_id() >= (unsigned)o) x += y;
        }
        if (lane_id() == 31) tmp[threadIdx.x >> 5] = x;
        __syncthreads();
        uint32_t add = carry;
        for (unsigned w = 0; w < (threadIdx.x >> 5); ++w) add += tmp[w];
        if (i < tiles) col[i] = add + x - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = add + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        totals[pass * 256 + d] = carry;
        if (carry == n) skip[pass] = 1u;
    }
}

// Stable scatter of one tile for pass `pass`, at the offsets from the superblock
// sums or from k_tile_scan.
template <typename K>
__global__ void __launch_bounds__(kSortThreads, 4) k_onesweep(
    K* kb0, uint32_t* vb0, K* kb1, uint32_t* vb1, uint32_t n, int pass, const uint32_t* __restrict__ skip,
    uint32_t* __restrict__ sel, const uint32_t* __restrict__ offsets, const uint32_t* __restrict__ totals,
    uint32_t tiles, int* err, const uint32_t* __restrict__ sup, uint32_t sups,
    const uint32_t* __restrict__ key_of_value) {
    const bool from1 = sel[pass] != 0;
    const K* __restrict__ kin = from1 ? kb1 : kb0;
    const uint32_t* __restrict__ vin = from1 ? vb1 : vb0;
    K* __restrict__ kout = from1 ? kb0 : kb1;
    uint32_t* __restrict__ vout = from1 ? vb0 : vb1;
    const int shift = 8 * pass;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* whist = reinterpret_cast<uint32_t*>(smem);  // [warps][256]
    uint32_t* tcount = whist + kSortWarps * 256;           // [256]
    uint32_t* lstart = tcount + 256;                       // [256]
    uint32_t* goff = lstart + 256;                         // [256]
    uint32_t* misc = goff + 256;                           // [16]
    K* skeys = reinterpret_cast<K*>(misc + 16);            // [tile]
    uint32_t* svals = reinterpret_cast<uint32_t*>(skeys + kSortTile);

    const int tid = threadIdx.x;
    const unsigned lane = lane_id();
    const int warp = tid >> 5;
    const uint32_t tile = blockIdx.x;
    const uint32_t base = tile * (uint32_t)kSortTile;
    const uint32_t tile_n = min((uint32_t)kSortTile, n - base);
    // every global load of the tile is issued before any ranking work
    K key[kSortItems];
    uint32_t val[kSortItems];
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const uint32_t idx = (uint32_t)warp * (32 * kSortItems) + (uint32_t)i * 32 + lane;
        key[i] = idx < tile_n ? kin[base + idx] : (K)0;
    }
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const uint32_t idx = (uint32_t)warp * (32 * kSortItems) + (uint32_t)i * 32 + lane;
        val[i] = idx < tile_n ? vin[base + idx] : 0u;
    }
    // digit tid: its keys in the tiles before this one (toff) and in all (dtot)
    uint32_t toff, dtot;
    bool skipped;
    if (sup != nullptr) {
        // the superblock sums before this tile's superblock, then the
        // tiles before it in its own
        // (fixed-count predicated loops: every load is in flight at once)
        const uint32_t sb = tile / kSortSup;
        const uint32_t* sp = sup + (size_t)pass * sups * 256 + tid;
        uint32_t tot = 0, pre = 0;
        for (uint32_t j0 = 0; j0 < sups; j0 += 32) {
            uint32_t v[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = j0 + j < sups ? sp[(size_t)(j0 + j) * 256] : 0u;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                tot += v[j];
                pre += j0 + j < sb ? v[j] : 0u;
            }
        }
        const uint32_t* cp = offsets + (size_t)sb * kSortSup * 256 + tid;
        const uint32_t before = tile - sb * kSortSup;  // tiles of this superblock before this one
        {
            uint32_t v[kSortSup];
#pragma unroll
            for (int j = 0; j < kSortSup; ++j) v[j] = (uint32_t)j < before ? cp[j * 256] : 0u;
#pragma unroll
            for (int j = 0; j < kSortSup; ++j) pre += v[j];
        }
        toff = pre;
        dtot = tot;
        skipped = __syncthreads_or(tot == n) != 0;
    } else {
        toff = offsets[(size_t)tid * tiles + tile];
        dtot = totals[pass * 256 + tid];
        skipped = skip[pass] != 0;
    }
    // the next pass reads the buffer this one writes, unless this one is
    // skipped (a constant digit: nothing moves)
    if (blockIdx.x == 0 && threadIdx.x == 0) sel[pass + 1] = skipped ? sel[pass] : (sel[pass] ^ 1u);
    if (skipped) return;
    for (int i = tid; i < kSortWarps * 256; i += kSortThreads) whist[i] = 0;
    __syncthreads();

    uint32_t rk[kSortItems];
    uint32_t* wh = whist + warp * 256;
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const uint32_t idx = (uint32_t)warp * (32 * kSortItems) + (uint32_t)i * 32 + lane;
        const bool valid = idx < tile_n;
        const uint32_t d = (uint32_t)(key[i] >> shift) & 255u;
        const unsigned peers = digit_peers(d, valid);
        uint32_t prior = valid ? wh[d] : 0u;
        __syncwarp();
        if (valid && lane == (unsigned)(__ffs(peers) - 1)) wh[d] = prior + __popc(peers);
        __syncwarp();
        rk[i] = prior + __popc(peers & lt);
    }
    __syncthreads();
    {
        // digit tid: warp exclusive offsets and the tile's count
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            uint32_t c = whist[w * 256 + tid];
            whist[w * 256 + tid] = run;
            run += c;
        }
        tcount[tid] = run;
    }
    uint32_t my = tcount[tid];
    uint32_t ls = block_excl_scan_256(my, misc + 8);
    const uint32_t dbase = block_excl_scan_256(dtot, misc + 8);  // the digit's first output position
    lstart[tid] = ls;
    goff[tid] = dbase + toff - ls;  // modulo 2^32
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        uint32_t idx = (uint32_t)warp * (32 * kSortItems) + (uint32_t)i * 32 + lane;
        if (idx < tile_n) {
            uint32_t d = (uint32_t)(key[i] >> shift) & 255u;
            uint32_t lp = lstart[d] + wh[d] + rk[i];
            skeys[lp] = key[i];
            svals[lp] = val[i];
        }
    }
    __syncthreads();
    for (uint32_t j = tid; j < tile_n; j += kSortThreads) {
        K k = skeys[j];
        uint32_t d = (uint32_t)(k >> shift) & 255u;
        uint32_t dst = goff[d] + j;
        if (dst < n) {  // always true for consistent counts; checked rather than trusted
            const uint32_t v = svals[j];
            kout[dst] = key_of_value != nullptr ? (K)(v < n ? key_of_value[v] : 0u) : k;
            vout[dst] = v;
        } else {
            flag_status(err, DEV_BAD);
        }
    }
}

// ---------------------------------------------------------------------------
// Tie compaction (3-phase scan over 2048-element blocks)
// ---------------------------------------------------------------------------
constexpr int kCmpThreads = 256;
constexpr int kCmpItems = 8;
constexpr int kCmpBlock = kCmpThreads * kCmpItems;

__device__ __forceinline__ void tie_flags(const uint8_t* eq, uint32_t n, uint32_t i, uint32_t& act,
                                          uint32_t& start) {
    uint32_t e = eq[i];
    uint32_t e1 = (i + 1 < n) ? eq[i + 1] : 0u;
    act = (e | e1) ? 1u : 0u;
    start = (act && !e) ? 1u : 0u;
}

__global__ void __launch_bounds__(kCmpThreads) k_tie_count(const uint8_t* __restrict__ eq,
                                                           uint32_t n, uint64_t* block_sums) {
    __shared__ uint32_t sa[kCmpThreads / 32], ss[kCmpThreads / 32];
    uint32_t a = 0, s = 0;
    uint32_t b0 = blockIdx.x * kCmpBlock;
    for (int j = 0; j < kCmpItems; ++j) {
        uint32_t i = b0 + j * kCmpThreads + threadIdx.x;
        if (i < n) {
            uint32_t x, y;
            tie_flags(eq, n, i, x, y);
            a += x;
            s += y;
        }
    }
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if (lane_id() == 0) {
        sa[threadIdx.x >> 5] = a;
        ss[threadIdx.x >> 5] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t ta = 0, ts = 0;
        for (int w = 0; w < kCmpThreads / 32; ++w) {
            ta += sa[w];
            ts += ss[w];
        }
        block_sums[blockIdx.x] = ((uint64_t)ta << 32) | ts;
    }
}

// Single CTA: exclusive scan of block sums in place; totals to total[0..1].
__global__ void __launch_bounds__(1024) k_scan_block_sums(uint64_t* sums, uint32_t nb,
                                                          uint32_t* total) {
    __shared__ uint64_t tmp[32];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t b0 = 0; b0 < nb; b0 += 1024) {
        uint32_t i = b0 + threadIdx.x;
        uint64_t v = i < nb ? sums[i] : 0ull;
        uint64_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane_id() >= (unsigned)o) x += y;
        }
        if (lane_id() == 31) tmp[threadIdx.x >> 5] = x;
        __syncthreads();
        uint64_t add = carry;
        for (unsigned w = 0; w < (threadIdx.x >> 5); ++w) add += tmp[w];
        if (i < nb) sums[i] = add + x - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = add + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        total[0] = (uint32_t)(carry >> 32);
        total[1] = (uint32_t)carry;
    }
}

__global__ void __launch_bounds__(kCmpThreads) k_tie_scatter(const uint8_t* __restrict__ eq,
                                                             uint32_t n,
                                                             const uint64_t* __restrict__ offs,
                                                             uint32_t* __restrict__ out_idx,
                                                             uint32_t* __restrict__ out_grp) {
    __shared__ uint64_t tmp[kCmpThreads / 32];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = offs[blockIdx.x];
    __syncthreads();
    uint32_t b0 = blockIdx.x * kCmpBlock;
    for (int j = 0; j < kCmpItems; ++j) {
        uint32_t i = b0 + j * kCmpThreads + threadIdx.x;
        uint32_t a = 0, s = 0;
        if (i < n) tie_flags(eq, n, i, a, s);
        uint64_t v = ((uint64_t)a << 32) | s;
        uint64_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane_id() >= (unsigned)o) x += y;
        }
        if (lane_id() == 31) tmp[threadIdx.x >> 5] = x;
        __syncthreads();
        uint64_t add = carry;
        for (unsigned w = 0; w < (threadIdx.x >> 5); ++w) add += tmp[w];
        uint64_t incl = add + x;
        if (a) {
            uint32_t slot = (uint32_t)((incl - v) >> 32);
            out_idx[slot] = i;
            out_grp[slot] = (uint32_t)incl - 1u;  // inclusive start count - 1
        }
        __syncthreads();
        if (threadIdx.x == kCmpThreads - 1) carry = incl;
        __syncthreads();
    }
}

}  // namespace lcpk

namespace lcph {
using namespace lcpk;

// Small pinned host buffer for the few counts the host reads back during a
// sort, allocated once per process per thread (cudaFreeHost would synchronise
// the whole device, so it is never freed per build).
uint32_t* pinned_words() {
    static thread_local uint32_t* buf = nullptr;
    if (!buf && cudaMallocHost((void**)&buf, sizeof(uint32_t) * 16) != cudaSuccess) buf = nullptr;
    return buf;
}

static void sort_work_carve(SortWork& w, uint32_t cap, Carver& c) {
    uint32_t tiles = (cap + kSortTile - 1) / kSortTile;
    uint32_t nb = (cap + kCmpBlock - 1) / kCmpBlock;
    if (tiles == 0) tiles = 1;
    if (nb == 0) nb = 1;
    const uint32_t sups = (tiles + kSortSup - 1) / kSortSup;
    w.sups = sups <= (uint32_t)kSortMaxSups ? sups : 0u;
    c.add(&w.hist, (size_t)kMaxPasses * 256);
    c.add(&w.skip, kMaxPasses);  // skip, sel and sup are zeroed together
    c.add(&w.sel, kMaxPasses + 1);
    if (w.sups) c.add(&w.sup, (size_t)kMaxPasses * 256 * w.sups);
    c.add(&w.status, (size_t)tiles * 256);
    c.add(&w.block_sums, nb);
    c.add(&w.total, 16);
}

int sort_work_alloc(SortWork& w, uint32_t cap, int* err, cudaStream_t s) {
    w.cap = cap;
    w.err = err;
    Carver c;
    sort_work_carve(w, cap, c);
    LCP_CUDA_TRY(c.alloc(&w.arena, s));
    w.h_total = pinned_words();
    if (!w.h_total) return LCP_ERR_OOM;
    return LCP_OK;
}

size_t sort_work_bytes(uint32_t cap) {
    SortWork w;
    Carver c;
    sort_work_carve(w, cap, c);
    return c.total;
}

int sort_work_place(SortWork& w, uint32_t cap, int* err, void* base) {
    w.cap = cap;
    w.err = err;
    Carver c;
    sort_work_carve(w, cap, c);
    c.place(base);
    w.arena = nullptr;  // not owned
    w.h_total = pinned_words();
    if (!w.h_total) return LCP_ERR_OOM;
    return LCP_OK;
}

void sort_work_free(SortWork& w, cudaStream_t s) {
    if (w.arena) cudaFreeAsync(w.arena, s);
    w = SortWork();
}

// Sync-free LSD radix sort: the result always ends in buffers 0.
template <typename K>
static int radix_sort_impl(K* k0, uint32_t* v0, K* k1, uint32_t* v1, uint32_t n, int key_bits,
                           SortWork& w, cudaStream_t s, K** out_k, uint32_t** out_v,
                           const uint32_t* key_of_value) {
    *out_k = k0;
    *out_v = v0;
    if (n <= 1) {
        if (n == 1 && key_of_value != nullptr) {  // the one key still maps
            LCP_CUDA_TRY(cudaMemsetAsync(w.sel, 0, sizeof(uint32_t) * 2, s));
            LCP_TIMED_LAUNCH(k_result_to_buf0<K>, 1, 32, 0, s, w.sel, 1, k1, v1, k0, v0, n, key_of_value);
        }
        return LCP_OK;
    }
    if (n > w.cap) return LCP_ERR_INVALID;
    int passes = (key_bits + 7) / 8;
    if (passes > (int)(sizeof(K))) passes = (int)sizeof(K);
    if (passes < 1) return LCP_OK;
    // no upfront histogram: each pass's digit totals come out of its own
    // counts (superblock sums, or the tile scan of a larger sort), and
    // constant digits are detected there
    const uint32_t tiles = (n + kSortTile - 1) / kSortTile;
    const uint32_t sups = (tiles + kSortSup - 1) / kSortSup;
    const bool fused = w.sup != nullptr && sups <= w.sups;
    {
        char* z0 = reinterpret_cast<char*>(w.skip);
        char* z1 = fused ? reinterpret_cast<char*>(w.sup + (size_t)passes * 256 * sups)
                         : reinterpret_cast<char*>(w.sel + kMaxPasses + 1);
        LCP_CUDA_TRY(cudaMemsetAsync(z0, 0, (size_t)(z1 - z0), s));
    }
    const size_t smem = sizeof(uint32_t) * (kSortWarps * 256 + 3 * 256 + 16) +
                        (sizeof(K) + sizeof(uint32_t)) * kSortTile;
    LCP_CUDA_TRY(cudaFuncSetAttribute(k_onesweep<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    uint32_t* sup = fused ? w.sup : nullptr;
    const uint32_t nsup = fused ? sups : 0u;
    for (int p = 0; p < passes; ++p) {
        LCP_TIMED_LAUNCH(k_tile_counts<K>, tiles, kSortThreads, 0, s, k0, k1, n, p, w.skip, w.sel, w.status,
                         tiles, sup, nsup);
        if (!fused) LCP_TIMED_LAUNCH(k_tile_scan, 256, 1024, 0, s, p, w.skip, w.status, tiles, w.hist, n);
        LCP_TIMED_LAUNCH(k_onesweep<K>, tiles, kSortThreads, smem, s, k0, v0, k1, v1, n, p, w.skip, w.sel,
                         w.status, w.hist, tiles, w.err, sup, nsup, p == passes - 1 ? key_of_value : nullptr);
    }
    unsigned cg = (unsigned)((n + 255) / 256);
    if (cg > (unsigned)sm_count() * 8) cg = sm_count() * 8;
    LCP_TIMED_LAUNCH(k_result_to_buf0<K>, cg, 256, 0, s, w.sel, passes, k1, v1, k0, v0, n, key_of_value);
    return LCP_OK;
}

int radix_sort_pairs_u64(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, uint32_t n,
                         int key_bits, SortWork& w, cudaStream_t s, uint64_t** out_k,
                         uint32_t** out_v) {
    return radix_sort_impl<uint64_t>(k0, v0, k1, v1, n, key_bits, w, s, out_k, out_v, nullptr);
}

int radix_sort_pairs_u32(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, uint32_t n,
                         int key_bits, SortWork& w, cudaStream_t s, uint32_t** out_k,
                         uint32_t** out_v, const uint32_t* key_of_value) {
    return radix_sort_impl<uint32_t>(k0, v0, k1, v1, n, key_bits, w, s, out_k, out_v, key_of_value);
}

int tie_compact_async(const uint8_t* eq, uint32_t n, uint32_t* out_idx, uint32_t* out_grp, SortWork& w,
                      cudaStream_t s) {
    if (n == 0) {
        LCP_CUDA_TRY(cudaMemsetAsync(w.total, 0, 2 * sizeof(uint32_t), s));
        return LCP_OK;
    }
    uint32_t nb = (n + kCmpBlock - 1) / kCmpBlock;
    LCP_TIMED_LAUNCH(k_tie_count, nb, kCmpThreads, 0, s, eq, n, w.block_sums);
    LCP_TIMED_LAUNCH(k_scan_block_sums, 1, 1024, 0, s, w.block_sums, nb, w.total);
    LCP_TIMED_LAUNCH(k_tie_scatter, nb, kCmpThreads, 0, s, eq, n, w.block_sums, out_idx, out_grp);
    return LCP_OK;
}

int tie_compact(const uint8_t* eq, uint32_t n, uint32_t* out_idx, uint32_t* out_grp,
                uint32_t* h_count, uint32_t* h_groups, SortWork& w, cudaStream_t s) {
    *h_count = 0;
    if (h_groups) *h_groups = 0;
    if (n == 0) return LCP_OK;
    int rc = tie_compact_async(eq, n, out_idx, out_grp, w, s);
    if (rc != LCP_OK) return rc;
    LCP_CUDA_TRY(cudaMemcpyAsync(w.h_total + 8, w.total, sizeof(uint32_t) * 2,
                                 cudaMemcpyDeviceToHost, s));
    LCP_CUDA_TRY(cudaStreamSynchronize(s));
    *h_count = w.h_total[8];
    if (h_groups) *h_groups = w.h_total[9];
    return LCP_OK;
}

}  // namespace lcph
