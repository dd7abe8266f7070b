/*
 * CPU oracle for LCP-based top-k retrieval -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the plain, slow, obviously correct statement of what the GPU
 * library computes.  It exists so that tests, the smoke check and the CPU
 * baseline leg of the benchmark can compare the CUDA path against it.  The
 * product path never links, loads or calls it, and it shares no code, header,
 * table or helper with the CUDA sources.
 *
 * Paper: "Optimal Space-Time Tradeoffs for LCP-Based Similarity Retrieval".
 *
 *   oracle_lcp          Definition "LCP Similarity" (Sec. 2.1): the largest j
 *                       with s[1..j] = t[1..j]; 0 when the first symbols differ.
 *   oracle_topk         Definition "Top-k LCP Retrieval" (Sec. 2.1): the k items
 *                       with the highest LCP to q, ties broken by (ascending,
 *                       0-based) original index.  Written as: LCP against every
 *                       stored sequence, then a stable sort of 0..N-1 on the key
 *                       (-LCP).  The stable sort is a counting sort over the LCP
 *                       value (a textbook stable sort), so equal LCPs keep index
 *                       order.  When k > N the tail is padded with (id -1, lcp 0).
 *   oracle_topk_batch   The same, for a batch of queries, split over threads (the
 *                       per-query computation is unchanged).
 *   oracle_topk_bfs     Algorithms 3 + 4 taken literally (the paper's own output
 *                       order, a variant): descend to the deepest node v on q's
 *                       path -- its depth d is the largest LCP of q with any
 *                       stored sequence -- and return the first k items of the
 *                       subtree T_v in BFS order.  With every sequence of the
 *                       same length L, items sit only at depth-L leaves, BFS
 *                       meets those leaves in lexicographic order, and a leaf's
 *                       posting list is in index order: so the answer is the
 *                       items with LCP == d, sorted by (sequence, index), cut
 *                       at k (fewer when |T_v| < k), each with LCP d.
 *   oracle_tal_topk     Thermal-Aware Logic (Definition "TAL", Sec. 6.2 and the
 *                       TALRangeScan listing, App. D): the bucket is the items
 *                       sharing q's first d symbols; only the bucket is scanned
 *                       and its top k by the Definition "Top-k LCP Retrieval"
 *                       order are returned (fewer when the bucket holds fewer).
 *   oracle_topk_wide    Definition "Top-k LCP Retrieval" for rows of any length
 *   (+ _batch)          1 <= L <= 65535, with 16-bit LCP values: the paper's
 *                       sustained benchmark (Sec. 7, Table 4; the sustained-load
 *                       configuration of App. C) stores sequences of max_len 256,
 *                       whose LCP with a query reaches 256.  The same steps as
 *                       oracle_topk (LCP against every sequence, counting sort on
 *                       -LCP over 0..L, first k), with the counts sized to L.
 *   oracle_sorted_index_wide  oracle_sorted_index for any L, H in 16 bits.
 *   oracle_sorted_index The array form of the trie built by Algorithm 1
 *                       (BuildLCPIndex, Sec. 5.2): item indices ordered by their
 *                       sequence (unsigned lexicographic order of the tokens;
 *                       equal sequences by index, the order in which Algorithm 1
 *                       appends them to a posting list), and the adjacent-LCP
 *                       array H[p] = LCP(row p-1, row p), H[0] = 0.  Sorting uses
 *                       the C library's qsort with an explicit comparator.
 *
 * Tokens are unsigned integers stored row-major, token_bytes = 1 (uint8) or 2
 * (uint16) per token, L tokens per sequence.
 *
 * Parity is pinned by tests that do not reuse this code: exhaustive enumeration
 * on tiny alphabets, a pointer trie that follows Algorithms 1-4 literally,
 * Python's own sort and os.path.commonprefix, the ultrametric property
 * (Theorem 1), the descent lemma (App. A), and a hand-worked example.
 */
#define _GNU_SOURCE
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Token i of a row (0-based position). */
static unsigned tok(const void* row, int64_t i, int token_bytes) {
    if (token_bytes == 1) return ((const uint8_t*)row)[i];
    return ((const uint16_t*)row)[i];
}

static const void* row_ptr(const void* base, int64_t r, int L, int token_bytes) {
    return (const uint8_t*)base + (size_t)r * (size_t)L * (size_t)token_bytes;
}

/* Definition "LCP Similarity": count matching leading symbols. */
int oracle_lcp(const void* s, const void* t, int L, int token_bytes) {
    int j = 0;
    while (j < L && tok(s, j, token_bytes) == tok(t, j, token_bytes)) j++;
    return j;
}

/*
 * Definition "Top-k LCP Retrieval" for one query.
 *   S: N rows of L tokens; q: one row; k >= 1.
 *   out_ids[k], out_lcp[k]: result rows in order (LCP descending, id ascending),
 *   padded with (-1, 0) beyond min(k, N).
 * lcp_buf (N ints) and order_buf (N ints) are caller-provided work arrays.
 * Returns 0, or -1 on bad arguments.
 */
int oracle_topk_work(const void* S, int64_t N, int L, int token_bytes, const void* q,
                     int k, int32_t* out_ids, uint8_t* out_lcp, int* lcp_buf,
                     int32_t* order_buf) {
    if (k < 1 || L < 1 || L > 255 || (token_bytes != 1 && token_bytes != 2) || N < 0)
        return -1;
    /* LCP of q with every stored sequence. */
    for (int64_t i = 0; i < N; i++)
        lcp_buf[i] = oracle_lcp(row_ptr(S, i, L, token_bytes), q, L, token_bytes);
    /* Stable counting sort of the indices 0..N-1 by descending LCP. */
    int64_t count[257];
    int64_t start[257];
    memset(count, 0, sizeof(count));
    for (int64_t i = 0; i < N; i++) count[lcp_buf[i]]++;
    int64_t acc = 0;
    for (int v = L; v >= 0; v--) {
        start[v] = acc;
        acc += count[v];
    }
    for (int64_t i = 0; i < N; i++) order_buf[start[lcp_buf[i]]++] = (int32_t)i;
    /* The first min(k, N) entries, then padding. */
    for (int r = 0; r < k; r++) {
        if (r < N) {
            out_ids[r] = order_buf[r];
            out_lcp[r] = (uint8_t)lcp_buf[order_buf[r]];
        } else {
            out_ids[r] = -1;
            out_lcp[r] = 0;
        }
    }
    return 0;
}

int oracle_topk(const void* S, int64_t N, int L, int token_bytes, const void* q, int k,
                int32_t* out_ids, uint8_t* out_lcp) {
    int* lcp_buf = (int*)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
    int32_t* order_buf = (int32_t*)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    if (!lcp_buf || !order_buf) {
        free(lcp_buf);
        free(order_buf);
        return -2;
    }
    int rc = oracle_topk_work(S, N, L, token_bytes, q, k, out_ids, out_lcp, lcp_buf,
                              order_buf);
    free(lcp_buf);
    free(order_buf);
    return rc;
}

/* ---- batch driver: queries split across threads, per-query work unchanged ---- */

typedef struct {
    const void* S;
    int64_t N;
    int L, token_bytes;
    const void* Qs;
    int64_t q_begin, q_end;
    int k;
    int32_t* out_ids;
    uint8_t* out_lcp;
    int rc;
} batch_job_t;

static void* batch_worker(void* arg) {
    batch_job_t* j = (batch_job_t*)arg;
    int* lcp_buf = (int*)malloc(sizeof(int) * (size_t)(j->N > 0 ? j->N : 1));
    int32_t* order_buf = (int32_t*)malloc(sizeof(int32_t) * (size_t)(j->N > 0 ? j->N : 1));
    j->rc = 0;
    if (!lcp_buf || !order_buf) {
        j->rc = -2;
    } else {
        for (int64_t qi = j->q_begin; qi < j->q_end && j->rc == 0; qi++) {
            j->rc = oracle_topk_work(j->S, j->N, j->L, j->token_bytes,
                                     row_ptr(j->Qs, qi, j->L, j->token_bytes), j->k,
                                     j->out_ids + (size_t)qi * (size_t)j->k,
                                     j->out_lcp + (size_t)qi * (size_t)j->k, lcp_buf,
                                     order_buf);
        }
    }
    free(lcp_buf);
    free(order_buf);
    return NULL;
}

int oracle_topk_batch(const void* S, int64_t N, int L, int token_bytes, const void* Qs,
                      int64_t Q, int k, int32_t* out_ids, uint8_t* out_lcp,
                      int n_threads) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    if (Q < (int64_t)n_threads) n_threads = (int)(Q > 0 ? Q : 1);
    batch_job_t jobs[256];
    pthread_t th[256];
    int64_t per = (Q + n_threads - 1) / n_threads;
    int started = 0;
    for (int t = 0; t < n_threads; t++) {
        jobs[t].S = S;
        jobs[t].N = N;
        jobs[t].L = L;
        jobs[t].token_bytes = token_bytes;
        jobs[t].Qs = Qs;
        jobs[t].q_begin = (int64_t)t * per;
        jobs[t].q_end = jobs[t].q_begin + per < Q ? jobs[t].q_begin + per : Q;
        jobs[t].k = k;
        jobs[t].out_ids = out_ids;
        jobs[t].out_lcp = out_lcp;
        jobs[t].rc = 0;
        if (pthread_create(&th[t], NULL, batch_worker, &jobs[t]) == 0) {
            started = t + 1;
        } else {
            batch_worker(&jobs[t]);
            started = t + 1;
            th[t] = 0;
        }
    }
    int rc = 0;
    for (int t = 0; t < started; t++) {
        if (th[t]) pthread_join(th[t], NULL);
        if (jobs[t].rc) rc = jobs[t].rc;
    }
    return rc;
}

/* ---- Algorithm 1 in array form: sorted order of the items, plus H ---- */

typedef struct {
    const void* S;
    int L, token_bytes;
} sort_ctx_t;

static int cmp_items(const void* a, const void* b, void* arg);

/*
 * Algorithms 3 + 4 for one query (see the header): out_ids[k], out_lcp[k],
 * padded with (-1, 0) beyond min(k, |T_v|).
 */
int oracle_topk_bfs(const void* S, int64_t N, int L, int token_bytes, const void* q, int k,
                    int32_t* out_ids, uint8_t* out_lcp) {
    if (k < 1 || L < 1 || L > 255 || (token_bytes != 1 && token_bytes != 2) || N < 0) return -1;
    int* lam = (int*)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
    int32_t* tv = (int32_t*)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    if (!lam || !tv) {
        free(lam);
        free(tv);
        return -2;
    }
    int d = 0;
    for (int64_t i = 0; i < N; i++) {
        lam[i] = oracle_lcp(row_ptr(S, i, L, token_bytes), q, L, token_bytes);
        if (lam[i] > d) d = lam[i];
    }
    int64_t n = 0;  /* T_v: the items whose LCP reaches the descent depth d */
    for (int64_t i = 0; i < N; i++)
        if (lam[i] == d) tv[n++] = (int32_t)i;
    sort_ctx_t c = {S, L, token_bytes};
    qsort_r(tv, (size_t)n, sizeof(int32_t), cmp_items, &c);
    for (int r = 0; r < k; r++) {
        out_ids[r] = r < n ? tv[r] : -1;
        out_lcp[r] = r < n ? (uint8_t)d : 0;
    }
    free(lam);
    free(tv);
    return 0;
}

/*
 * TAL for one query with prefix depth d (0 <= d <= L): the top k of the
 * bucket {i : LCP(S_i, q) >= d} by (LCP desc, index asc), padded.
 */
int oracle_tal_topk(const void* S, int64_t N, int L, int token_bytes, const void* q, int k, int d,
                    int32_t* out_ids, uint8_t* out_lcp) {
    if (k < 1 || L < 1 || L > 255 || d < 0 || d > L || (token_bytes != 1 && token_bytes != 2) || N < 0)
        return -1;
    int* lam = (int*)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
    if (!lam) return -2;
    for (int64_t i = 0; i < N; i++) lam[i] = oracle_lcp(row_ptr(S, i, L, token_bytes), q, L, token_bytes);
    int r = 0;
    /* LCP levels from L down to d; within a level, ascending index */
    for (int v = L; v >= d && r < k; v--)
        for (int64_t i = 0; i < N && r < k; i++)
            if (lam[i] == v) {
                out_ids[r] = (int32_t)i;
                out_lcp[r] = (uint8_t)v;
                r++;
            }
    for (; r < k; r++) {
        out_ids[r] = -1;
        out_lcp[r] = 0;
    }
    free(lam);
    return 0;
}

/* Unsigned lexicographic comparison of two stored rows, then by index. */
static int cmp_items(const void* a, const void* b, void* arg) {
    const sort_ctx_t* c = (const sort_ctx_t*)arg;
    int32_t ia = *(const int32_t*)a, ib = *(const int32_t*)b;
    const void* ra = row_ptr(c->S, ia, c->L, c->token_bytes);
    const void* rb = row_ptr(c->S, ib, c->L, c->token_bytes);
    for (int j = 0; j < c->L; j++) {
        unsigned x = tok(ra, j, c->token_bytes), y = tok(rb, j, c->token_bytes);
        if (x != y) return x < y ? -1 : 1;
    }
    return ia < ib ? -1 : (ia > ib ? 1 : 0);
}

/*
 * out_ids[N]: item indices in sorted order; out_H[N]: H[0] = 0 and
 * H[p] = LCP(S[out_ids[p-1]], S[out_ids[p]]).
 */
int oracle_sorted_index(const void* S, int64_t N, int L, int token_bytes,
                        int32_t* out_ids, uint8_t* out_H) {
    if (L < 1 || L > 255 || (token_bytes != 1 && token_bytes != 2) || N < 0) return -1;
    for (int64_t i = 0; i < N; i++) out_ids[i] = (int32_t)i;
    sort_ctx_t c = {S, L, token_bytes};
    qsort_r(out_ids, (size_t)N, sizeof(int32_t), cmp_items, &c);
    for (int64_t p = 0; p < N; p++) {
        out_H[p] = p == 0 ? 0
                          : (uint8_t)oracle_lcp(row_ptr(S, out_ids[p - 1], L, token_bytes),
                                                row_ptr(S, out_ids[p], L, token_bytes), L,
                                                token_bytes);
    }
    return 0;
}

/* ---- rows of any length: 16-bit LCP values (see the header) ---- */

/* count, start: L + 1 entries each (caller-provided work arrays). */
static int topk_wide_work(const void* S, int64_t N, int L, int token_bytes, const void* q, int k,
                          int32_t* out_ids, uint16_t* out_lcp, int* lcp_buf, int32_t* order_buf,
                          int64_t* count, int64_t* start) {
    for (int64_t i = 0; i < N; i++)
        lcp_buf[i] = oracle_lcp(row_ptr(S, i, L, token_bytes), q, L, token_bytes);
    memset(count, 0, sizeof(int64_t) * (size_t)(L + 1));
    for (int64_t i = 0; i < N; i++) count[lcp_buf[i]]++;
    int64_t acc = 0;
    for (int v = L; v >= 0; v--) {
        start[v] = acc;
        acc += count[v];
    }
    for (int64_t i = 0; i < N; i++) order_buf[start[lcp_buf[i]]++] = (int32_t)i;
    for (int r = 0; r < k; r++) {
        if (r < N) {
            out_ids[r] = order_buf[r];
            out_lcp[r] = (uint16_t)lcp_buf[order_buf[r]];
        } else {
            out_ids[r] = -1;
            out_lcp[r] = 0;
        }
    }
    return 0;
}

typedef struct {
    const void* S;
    int64_t N;
    int L, token_bytes;
    const void* Qs;
    int64_t q_begin, q_end;
    int k;
    int32_t* out_ids;
    uint16_t* out_lcp;
    int rc;
} wide_job_t;

static void* wide_worker(void* arg) {
    wide_job_t* j = (wide_job_t*)arg;
    int* lcp_buf = (int*)malloc(sizeof(int) * (size_t)(j->N > 0 ? j->N : 1));
    int32_t* order_buf = (int32_t*)malloc(sizeof(int32_t) * (size_t)(j->N > 0 ? j->N : 1));
    int64_t* count = (int64_t*)malloc(sizeof(int64_t) * (size_t)(j->L + 1));
    int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(j->L + 1));
    j->rc = 0;
    if (!lcp_buf || !order_buf || !count || !start) {
        j->rc = -2;
    } else {
        for (int64_t qi = j->q_begin; qi < j->q_end && j->rc == 0; qi++)
            j->rc = topk_wide_work(j->S, j->N, j->L, j->token_bytes, row_ptr(j->Qs, qi, j->L, j->token_bytes),
                                   j->k, j->out_ids + (size_t)qi * (size_t)j->k,
                                   j->out_lcp + (size_t)qi * (size_t)j->k, lcp_buf, order_buf, count, start);
    }
    free(lcp_buf);
    free(order_buf);
    free(count);
    free(start);
    return NULL;
}

/* Top-k of Q queries over rows of length 1 <= L <= 65535: out_ids [Q, k],
 * out_lcp [Q, k] uint16, padded with (-1, 0).  Queries split over threads. */
int oracle_topk_wide_batch(const void* S, int64_t N, int L, int token_bytes, const void* Qs, int64_t Q,
                           int k, int32_t* out_ids, uint16_t* out_lcp, int n_threads) {
    if (k < 1 || L < 1 || L > 65535 || (token_bytes != 1 && token_bytes != 2) || N < 0 || Q < 0) return -1;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    if (Q < (int64_t)n_threads) n_threads = (int)(Q > 0 ? Q : 1);
    wide_job_t jobs[256];
    pthread_t th[256];
    int64_t per = (Q + n_threads - 1) / n_threads;
    int started = 0;
    for (int t = 0; t < n_threads; t++) {
        jobs[t].S = S;
        jobs[t].N = N;
        jobs[t].L = L;
        jobs[t].token_bytes = token_bytes;
        jobs[t].Qs = Qs;
        jobs[t].q_begin = (int64_t)t * per;
        jobs[t].q_end = jobs[t].q_begin + per < Q ? jobs[t].q_begin + per : Q;
        jobs[t].k = k;
        jobs[t].out_ids = out_ids;
        jobs[t].out_lcp = out_lcp;
        jobs[t].rc = 0;
        if (pthread_create(&th[t], NULL, wide_worker, &jobs[t]) == 0) {
            started = t + 1;
        } else {
            wide_worker(&jobs[t]);
            started = t + 1;
            th[t] = 0;
        }
    }
    int rc = 0;
    for (int t = 0; t < started; t++) {
        if (th[t]) pthread_join(th[t], NULL);
        if (jobs[t].rc) rc = jobs[t].rc;
    }
    return rc;
}

/* oracle_sorted_index for 1 <= L <= 65535, H in 16 bits. */
int oracle_sorted_index_wide(const void* S, int64_t N, int L, int token_bytes, int32_t* out_ids,
                             uint16_t* out_H) {
    if (L < 1 || L > 65535 || (token_bytes != 1 && token_bytes != 2) || N < 0) return -1;
    for (int64_t i = 0; i < N; i++) out_ids[i] = (int32_t)i;
    sort_ctx_t c = {S, L, token_bytes};
    qsort_r(out_ids, (size_t)N, sizeof(int32_t), cmp_items, &c);
    for (int64_t p = 0; p < N; p++) {
        out_H[p] = p == 0 ? 0
                          : (uint16_t)oracle_lcp(row_ptr(S, out_ids[p - 1], L, token_bytes),
                                                 row_ptr(S, out_ids[p], L, token_bytes), L, token_bytes);
    }
    return 0;
}
