// Shared device/host helpers of the LCP library (sm_103a).
//
// Packed rows: token j of a row lands in 64-bit word j / tpw, most significant
// token first (tpw = 8 tokens per word for uint8, 4 for uint16), and the tail
// of the last word is zero.  Unsigned comparison of packed words is then the
// unsigned lexicographic order of the token strings, and the LCP of two rows
// is w * tpw + clz(a_w ^ b_w) / bits at their first differing word w (or L if
// none differs) -- Definition "LCP Similarity", Sec. 2.1.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lcp.h"

namespace lcpk {

// ---------------------------------------------------------------------------
// Row format
// ---------------------------------------------------------------------------
struct RowFmt {
    int tb;         // bytes per token (1 or 2)
    int L;          // tokens per row
    int W;          // packed words per row
    int tpw;        // tokens per packed word
    int bits;       // bits per token
    int row_bytes;  // L * tb
    int aligned8;   // rows start on 8-byte boundaries and hold whole words
};

inline RowFmt make_fmt(int tb, int L, const void* base) {
    RowFmt f;
    f.tb = tb;
    f.L = L;
    f.tpw = 8 / tb;
    f.bits = 8 * tb;
    f.W = (L + f.tpw - 1) / f.tpw;
    f.row_bytes = L * tb;
    f.aligned8 = ((reinterpret_cast<uintptr_t>(base) & 7) == 0) && (f.row_bytes % 8 == 0);
    return f;
}

__device__ __forceinline__ uint32_t load_tok(const uint8_t* row, int t, int tb) {
    return tb == 1 ? (uint32_t)row[t] : (uint32_t)reinterpret_cast<const uint16_t*>(row)[t];
}

// Reorders a little-endian 8-byte load into most-significant-token-first.
__device__ __forceinline__ uint64_t msb_first(uint64_t x, int tb) {
    uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
    uint32_t sel = tb == 2 ? 0x1032u : 0x0123u;
    uint32_t nhi = __byte_perm(lo, 0, sel);
    uint32_t nlo = __byte_perm(hi, 0, sel);
    return ((uint64_t)nhi << 32) | nlo;
}

// Packed word w of the raw row starting at `row`.
__device__ __forceinline__ uint64_t pack_word(const uint8_t* row, int w, const RowFmt& f) {
    if (f.aligned8) {
        uint64_t x = __ldg(reinterpret_cast<const unsigned long long*>(row) + w);
        return msb_first(x, f.tb);
    }
    uint64_t r = 0;
    int t0 = w * f.tpw;
#pragma unroll 1
    for (int j = 0; j < f.tpw; ++j) {
        int t = t0 + j;
        uint32_t v = t < f.L ? load_tok(row, t, f.tb) : 0u;
        r = (r << f.bits) | v;
    }
    return r;
}

__device__ __forceinline__ const uint8_t* row_of(const void* base, int64_t r, const RowFmt& f) {
    return reinterpret_cast<const uint8_t*>(base) + (size_t)r * (size_t)f.row_bytes;
}

// LCP contribution of the first differing word (x = a ^ b != 0) at word w.
__device__ __forceinline__ int lcp_at(int w, uint64_t x, const RowFmt& f) {
    int l = w * f.tpw + (__clzll((long long)x) / f.bits);
    return l < f.L ? l : f.L;
}

// ---------------------------------------------------------------------------
// Warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---------------------------------------------------------------------------
// Bulk copies global -> shared memory by the TMA unit (cp.async.bulk), with
// completion counted on a shared-memory mbarrier.  Addresses must be 16-byte
// aligned and sizes multiples of 16 bytes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Makes initialised barriers (and earlier shared-memory accesses of this
// thread) visible to the asynchronous proxy before a bulk copy uses them.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// One arrival that also announces `bytes` of incoming bulk-copy data.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    uint64_t state;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
                 : "=l"(state)
                 : "r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    (void)state;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// Waits for the barrier's phase of the given parity to complete, at most
// `limit` polls; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
    const uint32_t a = smem_u32(bar);
    for (long long i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Device status codes written by kernels into a status word (0 = fine).
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BAD = 2 };

__device__ __forceinline__ void flag_status(int* status, int code) {
    if (status) atomicMax(status, code);
}

// Upper bound on spins of any device-side wait (each spin is at least one
// global load, so this is well under a second on B300).
constexpr long long kSpinLimit = 1ll << 24;

}  // namespace lcpk

// ---------------------------------------------------------------------------
// Host side: launch accounting and error plumbing (defined in abi.cu).
// ---------------------------------------------------------------------------
namespace lcph {
void count_launch(int n = 1);
int cuda_status(cudaError_t e);  // maps to LCP_ERR_* and records the last error text
int* lib_status_word();          // device pointer to the library-wide status word
int* lib_status_word_if_any();   // the same if it was allocated already, else null
int sm_count();                  // multiprocessors of the current device (cached)
// Optional per-kernel timing (lcp_kernel_timing): CUDA events recorded on the
// launching stream around the kernel; off by default and inside graph capture.
bool ktime_on();
void* ktime_begin(const char* name, cudaStream_t s);
void ktime_end(void* token, cudaStream_t s);
}  // namespace lcph

namespace lcph {
// Carves many device buffers out of one stream-ordered allocation: one
// allocator call (and one free) instead of one per buffer.  Every buffer
// starts on a 256-byte boundary.
struct Carver {
    struct Req {
        void** p;
        size_t bytes;
    };
    Req reqs[64];
    int n = 0;
    size_t total = 0;
    template <typename T>
    void add(T** p, size_t count) {
        const size_t b = (sizeof(T) * (count ? count : 1) + 255) & ~(size_t)255;
        reqs[n++] = {reinterpret_cast<void**>(p), b};
        total += b;
    }
    // Points the buffers into caller-provided memory of at least `total` bytes.
    void place(void* base) {
        char* c = static_cast<char*>(base);
        for (int i = 0; i < n; ++i) {
            *reqs[i].p = c;
            c += reqs[i].bytes;
        }
    }
    cudaError_t alloc(void** base, cudaStream_t s) {
        cudaError_t e = cudaMallocAsync(base, total ? total : 256, s);
        if (e != cudaSuccess) return e;
        char* c = static_cast<char*>(*base);
        for (int i = 0; i < n; ++i) {
            *reqs[i].p = c;
            c += reqs[i].bytes;
        }
        return cudaSuccess;
    }
};
}  // namespace lcph

#define LCP_LAUNCH(kern, grid, block, smem, stream, ...)                 \
    do {                                                                 \
        kern<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);        \
        lcph::count_launch();                                            \
    } while (0)

// LCP_LAUNCH with per-kernel event timing when it is switched on.
#define LCP_TIMED_LAUNCH(kern, grid, block, smem, stream, ...)                         \
    do {                                                                               \
        void* _tk = lcph::ktime_on() ? lcph::ktime_begin(#kern, (stream)) : nullptr;   \
        LCP_LAUNCH(kern, grid, block, smem, stream, __VA_ARGS__);                      \
        if (_tk) lcph::ktime_end(_tk, (stream));                                       \
    } while (0)

#define LCP_CUDA_TRY(expr)                                \
    do {                                                  \
        cudaError_t _e = (expr);                          \
        if (_e != cudaSuccess) return lcph::cuda_status(_e); \
    } while (0)
