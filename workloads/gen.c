/*
 * Fast path of the Zipf prefix-conditioned generator in workloads/__init__.py
 * (same definitions, bit for bit; the numpy version is the reference and a
 * test checks the two agree).  Input generation only: no retrieval arithmetic.
 */
#include <pthread.h>
#include <stdint.h>

static inline uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline double unif(uint64_t ka, int64_t j) {
    uint64_t z = splitmix64(ka ^ ((uint64_t)j * 0xD6E8FEB86659FD93ull));
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

/* first index with cdf[i] > u, clamped to V-1 (numpy searchsorted side=right) */
static inline int64_t rank0(const double* cdf, int64_t V, double u) {
    int64_t lo = 0, hi = V;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (cdf[mid] > u) hi = mid;
        else lo = mid + 1;
    }
    return lo < V ? lo : V - 1;
}

static inline uint16_t perm_token(uint64_t h, int64_t r0, int64_t V) {
    uint64_t a = splitmix64(h) | 1ull;
    uint64_t b = splitmix64(h ^ 0xD1B54A32D192ED03ull);
    return (uint16_t)((a * (uint64_t)r0 + b) & (uint64_t)(V - 1));
}

typedef struct {
    uint16_t* out;
    const uint16_t* S;
    const int64_t* src;
    const int64_t* cut;
    int64_t begin, end, L, V, item_offset;
    const double* cdf;
    uint64_t key, h0;
} job_t;

static void* run(void* p) {
    job_t* J = (job_t*)p;
    for (int64_t i = J->begin; i < J->end; ++i) {
        uint64_t ka = splitmix64(J->key + (uint64_t)(J->item_offset + i));
        uint64_t h = J->h0;
        int64_t c = J->cut ? J->cut[i] : 0;
        for (int64_t j = 0; j < J->L; ++j) {
            uint16_t t;
            if (j < c) t = J->S[J->src[i] * J->L + j];
            else t = perm_token(h, rank0(J->cdf, J->V, unif(ka, j)), J->V);
            J->out[i * J->L + j] = t;
            h = splitmix64(h ^ ((uint64_t)t + 1ull));
        }
    }
    return 0;
}

/* Rows (src == NULL) or queries (copies of S[src[i]] up to cut[i], then drawn). */
void gen_zipf_prefix(uint16_t* out, int64_t n, int64_t L, int64_t V, const double* cdf, uint64_t key,
                     uint64_t h0, int64_t item_offset, const uint16_t* S, const int64_t* src,
                     const int64_t* cut, int threads) {
    if (threads < 1) threads = 1;
    if (threads > 64) threads = 64;
    pthread_t th[64];
    job_t jobs[64];
    int64_t per = (n + threads - 1) / threads;
    for (int t = 0; t < threads; ++t) {
        jobs[t] = (job_t){out, S, src, cut, t * per, (t + 1) * per < n ? (t + 1) * per : n,
                          L, V, item_offset, cdf, key, h0};
        if (jobs[t].begin > jobs[t].end) jobs[t].begin = jobs[t].end;
        pthread_create(&th[t], 0, run, &jobs[t]);
    }
    for (int t = 0; t < threads; ++t) pthread_join(th[t], 0);
}
