// Full scan top-k: LCP of every query against all N rows (the paper's "full
// scan" baseline, Sec. 7), no index.
//
//   k_pack_plane0   word 0 of every row, packed, into one contiguous plane
//                   (8 bytes a row: 16 MB at N=2M, so it stays in L2 while
//                   thousands of query tiles stream over it).
//   k_scan_partial  grid = (query tiles) x (N slices); a thread owns one query
//                   and a max-heap of its k best keys (255-LCP)<<32 | id for
//                   its slice.  Rows arrive in increasing id, so a row can
//                   only enter a full heap with a strictly larger LCP than the
//                   heap's worst; that test is a masked XOR on word 0 (the
//                   first worst+1 tokens equal), and only rows passing it pay
//                   for an exact LCP over the remaining words.
//   k_scan_merge    keys are unique, so the k smallest over a query's slice
//                   lists are order independent: sort G lists' keys in shared
//                   memory, keep k, repeat until one list is left, write out.
#include "common.cuh"

namespace lcpk {

constexpr int kScanTile = 2048;     // plane-0 words staged per smem tile
constexpr int kMergeCap = 4096;     // keys sorted per merge CTA
constexpr uint64_t kKeyInf = ~0ull;

__global__ void k_pack_plane0(const uint8_t* __restrict__ tokens, RowFmt f, int64_t n,
                              uint64_t* __restrict__ plane0) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) plane0[i] = pack_word(row_of(tokens, i, f), 0, f);
}

__device__ __forceinline__ void heap_sift_down(uint64_t* h, int n, int i) {
    uint64_t v = h[i];
    for (;;) {
        int c = 2 * i + 1;
        if (c >= n) break;
        uint64_t cv = h[c];
        if (c + 1 < n) {
            uint64_t c2 = h[c + 1];
            if (c2 > cv) {
                cv = c2;
                ++c;
            }
        }
        if (cv <= v) break;
        h[i] = cv;
        i = c;
    }
    h[i] = v;
}

__device__ __forceinline__ void heap_push(uint64_t* h, int n, uint64_t v) {
    int i = n;
    while (i > 0) {
        int par = (i - 1) >> 1;
        uint64_t pv = h[par];
        if (pv >= v) break;
        h[i] = pv;
        i = par;
    }
    h[i] = v;
}

// Word-0 mask that tests "the first t tokens are equal" (t <= tpw).
__device__ __forceinline__ uint64_t prefix_mask(int t, int bits) {
    int b = t * bits;
    return b >= 64 ? ~0ull : (b == 0 ? 0ull : (~0ull << (64 - b)));
}

__global__ void __launch_bounds__(128) k_scan_partial(const uint8_t* __restrict__ tokens,
                                                      const uint64_t* __restrict__ plane0, RowFmt f,
                                                      int64_t N, const uint8_t* __restrict__ queries,
                                                      RowFmt qf, int64_t Q, int k, int64_t slice,
                                                      uint64_t* __restrict__ heaps) {
    __shared__ uint64_t tile[kScanTile];
    const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t s0 = (int64_t)blockIdx.y * slice;
    const int64_t s1 = s0 + slice < N ? s0 + slice : N;
    const bool active = qi < Q;
    const uint8_t* qrow = active ? row_of(queries, qi, qf) : nullptr;
    const uint64_t q0 = active ? pack_word(qrow, 0, qf) : 0;
    uint64_t* heap = heaps + ((int64_t)blockIdx.y * Q + (active ? qi : 0)) * k;
    int hn = 0;
    uint64_t mask = 0;      // rows failing ((r ^ q0) & mask) == 0 cannot enter
    int worst = -1;         // LCP of the heap's worst entry once full
    for (int64_t t0 = s0; t0 < s1; t0 += kScanTile) {
        const int tn = (int)(s1 - t0 < kScanTile ? s1 - t0 : kScanTile);
        __syncthreads();
        for (int j = threadIdx.x; j < tn; j += blockDim.x) tile[j] = plane0[t0 + j];
        __syncthreads();
        if (!active) continue;
#pragma unroll 4
        for (int j = 0; j < tn; ++j) {
            const uint64_t r = tile[j];
            if (((r ^ q0) & mask) != 0) continue;
            // exact LCP of row t0+j
            int lam;
            uint64_t x = r ^ q0;
            if (x) {
                lam = __clzll((long long)x) / f.bits;
            } else {
                lam = f.L;
                const uint8_t* row = row_of(tokens, t0 + j, f);
                for (int w = 1; w < f.W; ++w) {
                    uint64_t y = pack_word(row, w, f) ^ pack_word(qrow, w, qf);
                    if (y) {
                        lam = w * f.tpw + (__clzll((long long)y) / f.bits);
                        break;
                    }
                }
                if (lam > f.L) lam = f.L;
            }
            if (hn == k && lam <= worst) continue;
            const uint64_t key = ((uint64_t)(255 - lam) << 32) | (uint64_t)(t0 + j);
            if (hn < k) {
                heap_push(heap, hn, key);
                ++hn;
            } else {
                heap[0] = key;
                heap_sift_down(heap, hn, 0);
            }
            if (hn == k) {
                worst = 255 - (int)(heap[0] >> 32);
                int t = worst + 1;
                mask = t <= f.tpw ? prefix_mask(t, f.bits) : ~0ull;
            }
        }
    }
    if (active)
        for (int j = hn; j < k; ++j) heap[j] = kKeyInf;
}

// Reduces groups of G lists of k keys per query to one list each (sorted when
// `final`, which then writes ids and LCPs).  grid = (Q, groups).
__global__ void __launch_bounds__(256) k_scan_merge(const uint64_t* __restrict__ in, int64_t Q,
                                                    int k, int nlists, int G, int P,
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
            v = in[((int64_t)(l0 + l) * Q + q) * k + j];
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

}  // namespace lcpk

namespace lcph {
using namespace lcpk;

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
    const int threads = 128;
    const int64_t qtiles = (Q + threads - 1) / threads;
    const int64_t target = 148 * 8;
    int64_t S = (target + qtiles - 1) / qtiles;
    int64_t maxS = (N + 1023) / 1024;
    if (S > maxS) S = maxS;
    if (S > 65535) S = 65535;
    if (S < 1) S = 1;
    int64_t slice = (N + S - 1) / S;
    S = (N + slice - 1) / slice;
    uint64_t* plane0 = nullptr;
    uint64_t* heaps = nullptr;
    LCP_CUDA_TRY(cudaMallocAsync((void**)&plane0, sizeof(uint64_t) * N, s));
    LCP_CUDA_TRY(cudaMallocAsync((void**)&heaps, sizeof(uint64_t) * (size_t)S * Q * k, s));
    LCP_TIMED_LAUNCH(k_pack_plane0, (unsigned)((N + 255) / 256), 256, 0, s,
               reinterpret_cast<const uint8_t*>(d_tokens), f, N, plane0);
    dim3 grid((unsigned)qtiles, (unsigned)S);
    LCP_TIMED_LAUNCH(k_scan_partial, grid, threads, 0, s, reinterpret_cast<const uint8_t*>(d_tokens),
               plane0, f, N, reinterpret_cast<const uint8_t*>(d_queries), qf, Q, k, slice, heaps);
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
        LCP_TIMED_LAUNCH(k_scan_merge, mg, 256, smem, s, cur, Q, k, (int)nl, g, P, out,
                   final_pass ? 1 : 0, d_out_ids, d_out_lcp);
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
