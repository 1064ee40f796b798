/*
 * nw_oracle.c -- plain CPU oracle for all-pairs Needleman-Wunsch scoring.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * definition that the CUDA library is checked against.  Only the test suite,
 * the package smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header or table with the CUDA library.
 *
 * What it computes (arxiv 2509.01654):
 *   - nwo_score_matrix / nwo_score: Algorithm 1 ("Needleman-Wunsch") taken
 *     literally: an (len(A)+1) x (len(B)+1) int32 score matrix, first column
 *     p*i and first row p*j, every other cell the maximum of the diagonal
 *     value plus similarity(A[i-1], B[j-1]), the upper value plus p and the
 *     left value plus p; the result is the bottom-right cell (Section 2).
 *     similarity(a, b) is `match` when the codes are equal and `mismatch`
 *     otherwise, the paper's 1 / -1 matrix of Section 4 with free values.
 *   - nwo_all_pairs: every pair i < j in the row-major order of the upper
 *     triangle, (0,1), (0,2), ..., (n-2,n-1) (Section 4.1), so the entry of
 *     (i, j) sits at S_{i-1} + (j - i - 1) with S_{i-1} = i(2n - i - 1)/2
 *     elements before row i (Section 4.2, the sum S_r).
 *   - nwo_topk_rows / nwo_query_topk: for a word, all other words ranked by
 *     higher score first and lower index on equal scores; the first k kept.
 *     Edges are undirected (Section 4.1), so word i's neighbours come from
 *     both halves of the matrix; self pairs are excluded.
 *   - nwo_topk_rows_normalised: the same lists ranked by Section 5's
 *     length-normalised weight s / max(len(A), len(B)), compared exactly.
 *   - nwo_histogram: one bin per integer score, each unordered pair counted
 *     once (the edge-weight histogram of Section 5).
 *   - nwo_score_pairs: the scores of an explicit list of pairs.
 *   - the *_sim variants: the same with Algorithm 1's similarity read from a
 *     full alphabet x alphabet matrix instead of match / mismatch.
 *
 * Pins: every function above is checked by the oracle's own tests against
 * the paper's worked examples, brute-force enumeration of alignments, the
 * Levenshtein and LCS reductions, library sorts and counting identities.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NWO_OK 0
#define NWO_EINVAL -1
#define NWO_ENOMEM -2

static int32_t max3(int32_t a, int32_t b, int32_t c) {
    int32_t m = a > b ? a : b;
    return m > c ? m : c;
}

/* Algorithm 1 over a caller-provided (la+1)*(lb+1) matrix, row-major. */
int nwo_score_matrix(const uint8_t *A, int la, const uint8_t *B, int lb,
                     int match, int mismatch, int gap, int32_t *H) {
    if (la < 0 || lb < 0 || H == NULL) return NWO_EINVAL;
    const int w = lb + 1;
    for (int i = 0; i <= la; ++i) H[i * w + 0] = gap * i;
    for (int j = 0; j <= lb; ++j) H[0 * w + j] = gap * j;
    for (int i = 1; i <= la; ++i) {
        for (int j = 1; j <= lb; ++j) {
            int32_t cost = (A[i - 1] == B[j - 1]) ? match : mismatch;
            int32_t match_score = H[(i - 1) * w + (j - 1)] + cost;
            int32_t delete_score = H[(i - 1) * w + j] + gap;
            int32_t insert_score = H[i * w + (j - 1)] + gap;
            H[i * w + j] = max3(match_score, delete_score, insert_score);
        }
    }
    return NWO_OK;
}

static int32_t score_with(int32_t *buf, const uint8_t *A, int la, const uint8_t *B, int lb,
                          int match, int mismatch, int gap) {
    nwo_score_matrix(A, la, B, lb, match, mismatch, gap, buf);
    return buf[la * (lb + 1) + lb];
}

/* Algorithm 1 with a full similarity matrix (its similarity(A[i-1], B[j-1])
 * step read from sim[a * alphabet + b]; Section 2's matrix, which Section 6
 * proposes to tune per phoneme pair). */
int nwo_score_matrix_sim(const uint8_t *A, int la, const uint8_t *B, int lb, const int32_t *sim,
                         int alphabet, int gap, int32_t *H) {
    if (la < 0 || lb < 0 || H == NULL || sim == NULL) return NWO_EINVAL;
    const int w = lb + 1;
    for (int i = 0; i <= la; ++i) H[i * w + 0] = gap * i;
    for (int j = 0; j <= lb; ++j) H[0 * w + j] = gap * j;
    for (int i = 1; i <= la; ++i) {
        for (int j = 1; j <= lb; ++j) {
            int32_t cost = sim[(int)A[i - 1] * alphabet + (int)B[j - 1]];
            int32_t match_score = H[(i - 1) * w + (j - 1)] + cost;
            int32_t delete_score = H[(i - 1) * w + j] + gap;
            int32_t insert_score = H[i * w + (j - 1)] + gap;
            H[i * w + j] = max3(match_score, delete_score, insert_score);
        }
    }
    return NWO_OK;
}

int32_t nwo_score_sim(const uint8_t *A, int la, const uint8_t *B, int lb, const int32_t *sim, int alphabet,
                      int gap) {
    int32_t *H = (int32_t *)malloc(sizeof(int32_t) * (size_t)(la + 1) * (size_t)(lb + 1));
    if (!H) return INT32_MIN;
    nwo_score_matrix_sim(A, la, B, lb, sim, alphabet, gap, H);
    int32_t s = H[la * (lb + 1) + lb];
    free(H);
    return s;
}

int32_t nwo_score(const uint8_t *A, int la, const uint8_t *B, int lb, int match, int mismatch,
                  int gap) {
    int32_t *H = (int32_t *)malloc(sizeof(int32_t) * (size_t)(la + 1) * (size_t)(lb + 1));
    if (!H) return INT32_MIN;
    int32_t s = score_with(H, A, la, B, lb, match, mismatch, gap);
    free(H);
    return s;
}

/* ------------------------------------------------------------------------ */
/* threading: rows are dealt round-robin to a fixed number of threads       */

typedef struct {
    const uint8_t *codes;
    const uint32_t *offsets;
    uint32_t n;
    int match, mismatch, gap;
    int nthreads;
    int maxlen;
    /* job-specific */
    int32_t *all_out;
    const uint32_t *rows;
    uint32_t nrows;
    uint32_t k;
    uint32_t *top_idx;
    int32_t *top_score;
    const uint8_t *qcodes;
    const uint32_t *qoffsets;
    int qmaxlen;
    int32_t hist_lo;
    uint32_t nbins;
    int64_t *hist_parts; /* nthreads * nbins */
    int64_t *out_of_range;
    const uint32_t *pi, *pj;
    size_t npairs;
    const int32_t *sim; /* NULL: match / mismatch; else alphabet x alphabet */
    int alphabet;
    int failed; /* set by a worker whose scratch allocation failed */
} job_t;

/* a worker that could not allocate its scratch marks the job failed, so the
 * call reports NWO_ENOMEM instead of returning with rows unwritten */
static void worker_failed(job_t *J) { __atomic_store_n(&J->failed, 1, __ATOMIC_RELAXED); }

/* a pair's score under the job's similarity */
static int32_t score_job(const job_t *J, int32_t *H, const uint8_t *A, int la, const uint8_t *B, int lb) {
    if (J->sim) {
        nwo_score_matrix_sim(A, la, B, lb, J->sim, J->alphabet, J->gap, H);
        return H[la * (lb + 1) + lb];
    }
    return score_with(H, A, la, B, lb, J->match, J->mismatch, J->gap);
}

typedef struct {
    job_t *job;
    int tid;
    void (*fn)(job_t *, int);
} worker_t;

static void *run_worker(void *arg) {
    worker_t *w = (worker_t *)arg;
    w->fn(w->job, w->tid);
    return NULL;
}

static int run_threads(job_t *job, void (*fn)(job_t *, int)) {
    int T = job->nthreads < 1 ? 1 : job->nthreads;
    pthread_t *th = (pthread_t *)calloc((size_t)T, sizeof(pthread_t));
    worker_t *ws = (worker_t *)calloc((size_t)T, sizeof(worker_t));
    if (!th || !ws) { free(th); free(ws); return NWO_ENOMEM; }
    for (int t = 0; t < T; ++t) {
        ws[t].job = job; ws[t].tid = t; ws[t].fn = fn;
        if (t == 0) continue;
        if (pthread_create(&th[t], NULL, run_worker, &ws[t]) != 0) ws[t].fn = NULL;
    }
    fn(job, 0);
    for (int t = 1; t < T; ++t) {
        if (ws[t].fn) pthread_join(th[t], NULL);
        else fn(job, t); /* a thread that could not start: do its share here */
    }
    free(th); free(ws);
    return __atomic_load_n(&job->failed, __ATOMIC_RELAXED) ? NWO_ENOMEM : NWO_OK;
}

static int max_length(const uint32_t *offsets, uint32_t n) {
    uint32_t m = 0;
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t l = offsets[i + 1] - offsets[i];
        if (l > m) m = l;
    }
    return (int)m;
}

static int32_t *matrix_buffer(int la_max, int lb_max) {
    return (int32_t *)malloc(sizeof(int32_t) * (size_t)(la_max + 1) * (size_t)(lb_max + 1));
}

/* ------------------------------------------------------------------------ */
/* all pairs, row-major upper triangle                                       */

static void all_pairs_rows(job_t *J, int tid) {
    int32_t *H = matrix_buffer(J->maxlen, J->maxlen);
    if (!H) { worker_failed(J); return; }
    const uint64_t n = J->n;
    for (uint64_t i = (uint64_t)tid; i + 1 < n; i += (uint64_t)J->nthreads) {
        const uint8_t *A = J->codes + J->offsets[i];
        int la = (int)(J->offsets[i + 1] - J->offsets[i]);
        uint64_t row_start = i * (2 * n - i - 1) / 2; /* S_{i-1} */
        for (uint64_t j = i + 1; j < n; ++j) {
            const uint8_t *B = J->codes + J->offsets[j];
            int lb = (int)(J->offsets[j + 1] - J->offsets[j]);
            J->all_out[row_start + (j - i - 1)] =
                score_job(J, H, A, la, B, lb);
        }
    }
    free(H);
}

int nwo_all_pairs(const uint8_t *codes, const uint32_t *offsets, uint32_t n, int match,
                  int mismatch, int gap, int32_t *out, int nthreads) {
    if (!codes || !offsets || !out) return NWO_EINVAL;
    job_t J;
    memset(&J, 0, sizeof J);
    J.codes = codes; J.offsets = offsets; J.n = n;
    J.match = match; J.mismatch = mismatch; J.gap = gap;
    J.nthreads = nthreads < 1 ? 1 : nthreads;
    J.maxlen = max_length(offsets, n);
    J.all_out = out;
    return run_threads(&J, all_pairs_rows);
}

/* ------------------------------------------------------------------------ */
/* top-k neighbours                                                          */

/* true when (s1, j1) ranks before (s2, j2): higher score, then lower index */
static int ranks_before(int32_t s1, uint32_t j1, int32_t s2, uint32_t j2) {
    return s1 > s2 || (s1 == s2 && j1 < j2);
}

/* keep the k best seen so far in order; `cnt` entries are filled */
static void keep_best(uint32_t *idx, int32_t *sc, uint32_t k, uint32_t *cnt, int32_t s,
                      uint32_t j) {
    uint32_t c = *cnt;
    if (c == k && !ranks_before(s, j, sc[k - 1], idx[k - 1])) return;
    uint32_t pos = c < k ? c : k - 1; /* slot that receives the new entry */
    while (pos > 0 && ranks_before(s, j, sc[pos - 1], idx[pos - 1])) {
        sc[pos] = sc[pos - 1];
        idx[pos] = idx[pos - 1];
        --pos;
    }
    sc[pos] = s;
    idx[pos] = j;
    if (c < k) *cnt = c + 1;
}

static void topk_rows_worker(job_t *J, int tid) {
    int32_t *H = matrix_buffer(J->maxlen, J->maxlen);
    if (!H) { worker_failed(J); return; }
    for (uint32_t r = (uint32_t)tid; r < J->nrows; r += (uint32_t)J->nthreads) {
        uint32_t i = J->rows[r];
        const uint8_t *A = J->codes + J->offsets[i];
        int la = (int)(J->offsets[i + 1] - J->offsets[i]);
        uint32_t *idx = J->top_idx + (size_t)r * J->k;
        int32_t *sc = J->top_score + (size_t)r * J->k;
        uint32_t cnt = 0;
        for (uint32_t j = 0; j < J->n; ++j) {
            if (j == i) continue;
            const uint8_t *B = J->codes + J->offsets[j];
            int lb = (int)(J->offsets[j + 1] - J->offsets[j]);
            int32_t s = score_job(J, H, A, la, B, lb);
            keep_best(idx, sc, J->k, &cnt, s, j);
        }
        for (uint32_t c = cnt; c < J->k; ++c) { idx[c] = UINT32_MAX; sc[c] = INT32_MIN; }
    }
    free(H);
}

int nwo_topk_rows(const uint8_t *codes, const uint32_t *offsets, uint32_t n, const uint32_t *rows,
                  uint32_t nrows, uint32_t k, int match, int mismatch, int gap,
                  uint32_t *out_idx, int32_t *out_score, int nthreads) {
    if (!codes || !offsets || !rows || !out_idx || !out_score || k == 0) return NWO_EINVAL;
    for (uint32_t r = 0; r < nrows; ++r) if (rows[r] >= n) return NWO_EINVAL;
    job_t J;
    memset(&J, 0, sizeof J);
    J.codes = codes; J.offsets = offsets; J.n = n;
    J.match = match; J.mismatch = mismatch; J.gap = gap;
    J.nthreads = nthreads < 1 ? 1 : nthreads;
    J.maxlen = max_length(offsets, n);
    J.rows = rows; J.nrows = nrows; J.k = k;
    J.top_idx = out_idx; J.top_score = out_score;
    return run_threads(&J, topk_rows_worker);
}

/* Section 5's length normalisation: a pair's weight is s / max(len(A),
 * len(B)) (times 100 for display, which does not change the order).  Two empty
 * words have weight s / 1.  Weights are compared exactly, as fractions with
 * positive denominators: s1/m1 > s2/m2  <=>  s1*m2 > s2*m1. */
static int ranks_before_norm(int32_t s1, int32_t m1, uint32_t j1, int32_t s2, int32_t m2, uint32_t j2) {
    int64_t l = (int64_t)s1 * m2, r = (int64_t)s2 * m1;
    return l > r || (l == r && j1 < j2);
}

static void topk_rows_norm_worker(job_t *J, int tid) {
    int32_t *H = matrix_buffer(J->maxlen, J->maxlen);
    int32_t *den = (int32_t *)malloc(sizeof(int32_t) * J->k);
    if (!H || !den) { free(H); free(den); worker_failed(J); return; }
    for (uint32_t r = (uint32_t)tid; r < J->nrows; r += (uint32_t)J->nthreads) {
        uint32_t i = J->rows[r];
        const uint8_t *A = J->codes + J->offsets[i];
        int la = (int)(J->offsets[i + 1] - J->offsets[i]);
        uint32_t *idx = J->top_idx + (size_t)r * J->k;
        int32_t *sc = J->top_score + (size_t)r * J->k;
        uint32_t cnt = 0;
        for (uint32_t j = 0; j < J->n; ++j) {
            if (j == i) continue;
            const uint8_t *B = J->codes + J->offsets[j];
            int lb = (int)(J->offsets[j + 1] - J->offsets[j]);
            int32_t s = score_job(J, H, A, la, B, lb);
            int32_t m = la > lb ? la : lb;
            if (m == 0) m = 1;
            /* insertion into the ordered list, as keep_best but by weight */
            if (cnt == J->k && !ranks_before_norm(s, m, j, sc[J->k - 1], den[J->k - 1], idx[J->k - 1])) continue;
            uint32_t pos = cnt < J->k ? cnt : J->k - 1;
            while (pos > 0 && ranks_before_norm(s, m, j, sc[pos - 1], den[pos - 1], idx[pos - 1])) {
                sc[pos] = sc[pos - 1];
                den[pos] = den[pos - 1];
                idx[pos] = idx[pos - 1];
                --pos;
            }
            sc[pos] = s;
            den[pos] = m;
            idx[pos] = j;
            if (cnt < J->k) ++cnt;
        }
        for (uint32_t c = cnt; c < J->k; ++c) { idx[c] = UINT32_MAX; sc[c] = INT32_MIN; }
    }
    free(den);
    free(H);
}

/* As nwo_topk_rows, ranked by the normalised weight (ties: lower index);
 * out_score holds the raw scores s. */
int nwo_topk_rows_normalised(const uint8_t *codes, const uint32_t *offsets, uint32_t n, const uint32_t *rows,
                             uint32_t nrows, uint32_t k, int match, int mismatch, int gap,
                             uint32_t *out_idx, int32_t *out_score, int nthreads) {
    if (!codes || !offsets || !rows || !out_idx || !out_score || k == 0) return NWO_EINVAL;
    for (uint32_t r = 0; r < nrows; ++r) if (rows[r] >= n) return NWO_EINVAL;
    job_t J;
    memset(&J, 0, sizeof J);
    J.codes = codes; J.offsets = offsets; J.n = n;
    J.match = match; J.mismatch = mismatch; J.gap = gap;
    J.nthreads = nthreads < 1 ? 1 : nthreads;
    J.maxlen = max_length(offsets, n);
    J.rows = rows; J.nrows = nrows; J.k = k;
    J.top_idx = out_idx; J.top_score = out_score;
    return run_threads(&J, topk_rows_norm_worker);
}

static void query_worker(job_t *J, int tid) {
    int m = J->maxlen > J->qmaxlen ? J->maxlen : J->qmaxlen;
    int32_t *H = matrix_buffer(m, m);
    if (!H) { worker_failed(J); return; }
    for (uint32_t q = (uint32_t)tid; q < J->nrows; q += (uint32_t)J->nthreads) {
        const uint8_t *A = J->qcodes + J->qoffsets[q];
        int la = (int)(J->qoffsets[q + 1] - J->qoffsets[q]);
        uint32_t *idx = J->top_idx + (size_t)q * J->k;
        int32_t *sc = J->top_score + (size_t)q * J->k;
        uint32_t cnt = 0;
        for (uint32_t j = 0; j < J->n; ++j) {
            const uint8_t *B = J->codes + J->offsets[j];
            int lb = (int)(J->offsets[j + 1] - J->offsets[j]);
            int32_t s = score_job(J, H, A, la, B, lb);
            keep_best(idx, sc, J->k, &cnt, s, j);
        }
        for (uint32_t c = cnt; c < J->k; ++c) { idx[c] = UINT32_MAX; sc[c] = INT32_MIN; }
    }
    free(H);
}

/* every query against every dictionary word (a query is not a dictionary word,
 * so nothing is excluded) */
int nwo_query_topk(const uint8_t *qcodes, const uint32_t *qoffsets, uint32_t nq,
                   const uint8_t *codes, const uint32_t *offsets, uint32_t n, uint32_t k,
                   int match, int mismatch, int gap, uint32_t *out_idx, int32_t *out_score,
                   int nthreads) {
    if (!qcodes || !qoffsets || !codes || !offsets || !out_idx || !out_score || k == 0)
        return NWO_EINVAL;
    job_t J;
    memset(&J, 0, sizeof J);
    J.codes = codes; J.offsets = offsets; J.n = n;
    J.qcodes = qcodes; J.qoffsets = qoffsets; J.nrows = nq;
    J.match = match; J.mismatch = mismatch; J.gap = gap;
    J.nthreads = nthreads < 1 ? 1 : nthreads;
    J.maxlen = max_length(offsets, n);
    J.qmaxlen = max_length(qoffsets, nq);
    J.k = k; J.top_idx = out_idx; J.top_score = out_score;
    return run_threads(&J, query_worker);
}

/* ------------------------------------------------------------------------ */
/* histogram of all unordered pairs                                          */

static void histogram_rows(job_t *J, int tid) {
    int32_t *H = matrix_buffer(J->maxlen, J->maxlen);
    if (!H) { worker_failed(J); return; }
    int64_t *hist = J->hist_parts + (size_t)tid * J->nbins;
    int64_t bad = 0;
    for (uint32_t i = (uint32_t)tid; i + 1 < J->n; i += (uint32_t)J->nthreads) {
        const uint8_t *A = J->codes + J->offsets[i];
        int la = (int)(J->offsets[i + 1] - J->offsets[i]);
        for (uint32_t j = i + 1; j < J->n; ++j) {
            const uint8_t *B = J->codes + J->offsets[j];
            int lb = (int)(J->offsets[j + 1] - J->offsets[j]);
            int64_t b = (int64_t)score_job(J, H, A, la, B, lb) -
                        J->hist_lo;
            if (b < 0 || b >= (int64_t)J->nbins) ++bad; else ++hist[b];
        }
    }
    J->out_of_range[tid] = bad;
    free(H);
}

/* returns the number of pairs whose score fell outside [lo, lo + nbins), or <0 */
int64_t nwo_histogram(const uint8_t *codes, const uint32_t *offsets, uint32_t n, int match,
                      int mismatch, int gap, int32_t lo, uint32_t nbins, int64_t *hist,
                      int nthreads) {
    if (!codes || !offsets || !hist || nbins == 0) return NWO_EINVAL;
    job_t J;
    memset(&J, 0, sizeof J);
    J.codes = codes; J.offsets = offsets; J.n = n;
    J.match = match; J.mismatch = mismatch; J.gap = gap;
    J.nthreads = nthreads < 1 ? 1 : nthreads;
    J.maxlen = max_length(offsets, n);
    J.hist_lo = lo; J.nbins = nbins;
    J.hist_parts = (int64_t *)calloc((size_t)J.nthreads * nbins, sizeof(int64_t));
    J.out_of_range = (int64_t *)calloc((size_t)J.nthreads, sizeof(int64_t));
    if (!J.hist_parts || !J.out_of_range) { free(J.hist_parts); free(J.out_of_range); return NWO_ENOMEM; }
    int rc = run_threads(&J, histogram_rows);
    int64_t bad = 0;
    memset(hist, 0, sizeof(int64_t) * nbins);
    for (int t = 0; t < J.nthreads; ++t) {
        bad += J.out_of_range[t];
        for (uint32_t b = 0; b < nbins; ++b) hist[b] += J.hist_parts[(size_t)t * nbins + b];
    }
    free(J.hist_parts); free(J.out_of_range);
    return rc == NWO_OK ? bad : rc;
}

/* ------------------------------------------------------------------------ */
/* explicit pairs                                                            */

static void pairs_worker(job_t *J, int tid) {
    int32_t *H = matrix_buffer(J->maxlen, J->maxlen);
    if (!H) { worker_failed(J); return; }
    for (size_t p = (size_t)tid; p < J->npairs; p += (size_t)J->nthreads) {
        uint32_t i = J->pi[p], j = J->pj[p];
        J->all_out[p] = score_job(J, H, J->codes + J->offsets[i], (int)(J->offsets[i + 1] - J->offsets[i]),
                                  J->codes + J->offsets[j], (int)(J->offsets[j + 1] - J->offsets[j]));
    }
    free(H);
}

int nwo_score_pairs(const uint8_t *codes, const uint32_t *offsets, uint32_t n, const uint32_t *pi,
                    const uint32_t *pj, size_t m, int match, int mismatch, int gap, int32_t *out,
                    int nthreads) {
    if (!codes || !offsets || (m && (!pi || !pj || !out))) return NWO_EINVAL;
    for (size_t p = 0; p < m; ++p) if (pi[p] >= n || pj[p] >= n) return NWO_EINVAL;
    job_t J;
    memset(&J, 0, sizeof J);
    J.codes = codes; J.offsets = offsets; J.n = n;
    J.match = match; J.mismatch = mismatch; J.gap = gap;
    J.nthreads = nthreads < 1 ? 1 : nthreads;
    J.maxlen = max_length(offsets, n);
    J.pi = pi; J.pj = pj; J.npairs = m; J.all_out = out;
    return run_threads(&J, pairs_worker);
}

/* ------------------------------------------------------------------------ */
/* the same reductions under a full similarity matrix                       */

static int codes_below(const uint8_t *codes, const uint32_t *offsets, uint32_t n, int alphabet) {
    for (uint32_t x = offsets[0]; x < offsets[n]; ++x)
        if ((int)codes[x] >= alphabet) return 0;
    return 1;
}

static void sim_job(job_t *J, const uint8_t *codes, const uint32_t *offsets, uint32_t n, const int32_t *sim,
                    int alphabet, int gap, int nthreads) {
    memset(J, 0, sizeof *J);
    J->codes = codes; J->offsets = offsets; J->n = n;
    J->gap = gap;
    J->sim = sim; J->alphabet = alphabet;
    J->nthreads = nthreads < 1 ? 1 : nthreads;
    J->maxlen = max_length(offsets, n);
}

int nwo_all_pairs_sim(const uint8_t *codes, const uint32_t *offsets, uint32_t n, const int32_t *sim,
                      int alphabet, int gap, int32_t *out, int nthreads) {
    if (!codes || !offsets || !out || !sim || alphabet < 1) return NWO_EINVAL;
    if (!codes_below(codes, offsets, n, alphabet)) return NWO_EINVAL;
    job_t J;
    sim_job(&J, codes, offsets, n, sim, alphabet, gap, nthreads);
    J.all_out = out;
    return run_threads(&J, all_pairs_rows);
}

int nwo_topk_rows_sim(const uint8_t *codes, const uint32_t *offsets, uint32_t n, const uint32_t *rows,
                      uint32_t nrows, uint32_t k, const int32_t *sim, int alphabet, int gap,
                      uint32_t *out_idx, int32_t *out_score, int nthreads) {
    if (!codes || !offsets || !rows || !out_idx || !out_score || k == 0 || !sim || alphabet < 1) return NWO_EINVAL;
    for (uint32_t r = 0; r < nrows; ++r) if (rows[r] >= n) return NWO_EINVAL;
    if (!codes_below(codes, offsets, n, alphabet)) return NWO_EINVAL;
    job_t J;
    sim_job(&J, codes, offsets, n, sim, alphabet, gap, nthreads);
    J.rows = rows; J.nrows = nrows; J.k = k;
    J.top_idx = out_idx; J.top_score = out_score;
    return run_threads(&J, topk_rows_worker);
}

int64_t nwo_histogram_sim(const uint8_t *codes, const uint32_t *offsets, uint32_t n, const int32_t *sim,
                          int alphabet, int gap, int32_t lo, uint32_t nbins, int64_t *hist, int nthreads) {
    if (!codes || !offsets || !hist || nbins == 0 || !sim || alphabet < 1) return NWO_EINVAL;
    if (!codes_below(codes, offsets, n, alphabet)) return NWO_EINVAL;
    job_t J;
    sim_job(&J, codes, offsets, n, sim, alphabet, gap, nthreads);
    J.hist_lo = lo; J.nbins = nbins;
    J.hist_parts = (int64_t *)calloc((size_t)J.nthreads * nbins, sizeof(int64_t));
    J.out_of_range = (int64_t *)calloc((size_t)J.nthreads, sizeof(int64_t));
    if (!J.hist_parts || !J.out_of_range) { free(J.hist_parts); free(J.out_of_range); return NWO_ENOMEM; }
    int rc = run_threads(&J, histogram_rows);
    int64_t bad = 0;
    memset(hist, 0, sizeof(int64_t) * nbins);
    for (int t = 0; t < J.nthreads; ++t) {
        bad += J.out_of_range[t];
        for (uint32_t b = 0; b < nbins; ++b) hist[b] += J.hist_parts[(size_t)t * nbins + b];
    }
    free(J.hist_parts); free(J.out_of_range);
    return rc == NWO_OK ? bad : rc;
}

int nwo_score_pairs_sim(const uint8_t *codes, const uint32_t *offsets, uint32_t n, const uint32_t *pi,
                        const uint32_t *pj, size_t m, const int32_t *sim, int alphabet, int gap, int32_t *out,
                        int nthreads) {
    if (!codes || !offsets || (m && (!pi || !pj || !out)) || !sim || alphabet < 1) return NWO_EINVAL;
    for (size_t p = 0; p < m; ++p) if (pi[p] >= n || pj[p] >= n) return NWO_EINVAL;
    if (!codes_below(codes, offsets, n, alphabet)) return NWO_EINVAL;
    job_t J;
    sim_job(&J, codes, offsets, n, sim, alphabet, gap, nthreads);
    J.pi = pi; J.pj = pj; J.npairs = m; J.all_out = out;
    return run_threads(&J, pairs_worker);
}
