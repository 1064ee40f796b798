/*
 * nw.h -- C ABI of libnw: all-pairs Needleman-Wunsch scoring of phoneme-coded
 * words on one GB300 GPU (sm_103a).
 *
 * Method: arxiv 2509.01654, "Parallel Needleman-Wunsch on CUDA to measure word
 * similarity based on phonetic transcriptions".  A word is a sequence of
 * integer phoneme codes (Section 3, the encoding table); two words are scored
 * by the Needleman-Wunsch recurrence of Algorithm 1 with a similarity of
 * `match` for equal codes and `mismatch` otherwise and a gap value p added per
 * gap column (Section 2; Section 4 fixes match 1, mismatch -1, p = -1).  Edges
 * are undirected and self pairs are excluded, so only the upper triangle of
 * the word-by-word matrix is scored (Section 4.1).
 *
 * Conventions for every call:
 *  - Return value: NW_OK or a negative nw_status; a message for the last
 *    failure is available from nw_last_error().  The library never aborts,
 *    traps or exits.  On failure no output buffer has been partially written
 *    unless the message says otherwise.
 *  - Ownership: input buffers are borrowed for the duration of the call and
 *    copied; the library keeps no caller pointer.  Output buffers are
 *    allocated by the caller.
 *  - Host or device buffers: buffers are host memory unless the call's
 *    `flags` contain NW_DEVICE_PTRS, in which case every buffer argument of
 *    that call is a device pointer on the context's device.
 *  - Ordering: all GPU work is issued on the context's stream.  Calls return
 *    after that work has finished unless NW_ASYNC is given together with
 *    NW_DEVICE_PTRS, in which case outputs are valid once the stream reaches
 *    the point where the call returned.
 *  - Indices in results are the caller's original word indices.  Missing
 *    neighbours (fewer than k candidates) are reported as index UINT32_MAX
 *    and score INT16_MIN.
 *  - Thread safety: a context and its dictionaries are used by one host
 *    thread at a time; distinct contexts are independent.
 */
#ifndef NW_H
#define NW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Longest word accepted by the kernels (the paper's words have at most ~25
 * symbols, Section 4.1; queries and batched dictionaries go up to 40). */
#define NW_MAX_WORD_LEN 40
/* Largest neighbour-list length k. */
#define NW_MAX_K 128

typedef enum {
    NW_OK = 0,
    NW_EINVAL = -1,   /* invalid argument: null pointer, n < 2, k out of range, code >= alphabet, word too long, unsupported scoring */
    NW_ENOMEM = -2,   /* device allocation failed or the context's memory budget would be exceeded */
    NW_ERANGE = -3,   /* a score bound does not fit the output type, or nbins is too small */
    NW_ECUDA = -4,    /* a CUDA runtime error (message from the runtime in nw_last_error) */
    NW_ETIMEOUT = -5, /* a bounded device-side retry loop gave up; results are not valid */
    NW_EBUSY = -6     /* the context is in use by another call */
} nw_status;

/* call flags */
#define NW_DEVICE_PTRS 0x1u /* buffer arguments are device pointers */
#define NW_ASYNC 0x2u       /* with NW_DEVICE_PTRS: do not wait for the stream before returning */
#define NW_RANK_NORMALISED 0x4u /* nw_all_pairs_topk: rank neighbours by s / max(len) (Section 5) */

/* Similarity and gap values (Algorithm 1, Section 2): similarity(a, b) is
 * `match` when a == b and `mismatch` otherwise; `gap` (the paper's p, normally
 * negative) is added once per gap column.  The kernels require
 * mismatch <= match, 2*gap <= match and |match|, |mismatch|, |gap| <= 1024;
 * other values give NW_EINVAL. */
typedef struct {
    int32_t match;
    int32_t mismatch;
    int32_t gap;
} nw_scoring;

typedef struct nw_ctx nw_ctx;
typedef struct nw_dict nw_dict;

/* Facts about a loaded dictionary. */
typedef struct {
    uint32_t n;          /* words */
    uint32_t alphabet;   /* codes are < alphabet */
    uint32_t min_len, max_len;
    int32_t score_lo;    /* lowest score any pair of this dictionary can reach */
    int32_t score_hi;    /* highest score any pair can reach */
    uint32_t nbins;      /* score_hi - score_lo + 1: histogram bins nw_all_pairs_topk needs */
    uint32_t pad_;
    uint64_t pairs;      /* n(n-1)/2, the edge count of Section 4.2 */
    uint64_t cells;      /* sum over pairs of len(a)*len(b): DP cells of all pairs */
    uint64_t device_bytes; /* device memory held by the dictionary */
} nw_dict_info;

/* Timings of the last call, filled when profiling is enabled.  Durations come
 * from CUDA events recorded on the context's stream around each launch. */
typedef struct {
    double dp_ms;          /* summed duration of the alignment-kernel launches */
    double finalize_ms;    /* summed duration of the list-finalising launches */
    double total_ms;       /* first to last event of the call */
    uint32_t dp_launches;  /* alignment-kernel launches of the call */
    uint32_t launches;     /* all kernel launches of the call */
    uint64_t pairs;        /* pairs scored by the call */
    uint64_t cells;        /* DP cells of those pairs */
    uint64_t list_inserts; /* candidate neighbours that reached a global list */
} nw_profile;

/* Creates a context on CUDA device `device`.  `mem_budget_bytes` caps the
 * device memory the context may hold (0 = no cap); `cuda_stream` is a
 * cudaStream_t to issue work on, or NULL for a stream the context owns.  The
 * stream is borrowed and must outlive the context. */
nw_status nw_create(nw_ctx **out, int device, size_t mem_budget_bytes, void *cuda_stream);

/* Frees the context and every dictionary still loaded in it. */
void nw_destroy(nw_ctx *ctx);

/* Message for the last failed call on `ctx` ("" if none).  Valid until the
 * next call on the context.  With ctx == NULL: the message of the last failed
 * nw_create on this thread. */
const char *nw_last_error(const nw_ctx *ctx);

/* Turns per-call event timing on or off (off by default). */
nw_status nw_set_profiling(nw_ctx *ctx, int enable);

/* Copies the profile of the last call made with profiling on. */
nw_status nw_last_profile(const nw_ctx *ctx, nw_profile *out);

/* Loads a dictionary of n words given in CSR form: word i is
 * codes[offsets[i] .. offsets[i+1]), offsets has n+1 entries with
 * offsets[0] == 0, every code is < alphabet (alphabet <= 256) and every word
 * has at most NW_MAX_WORD_LEN codes (empty words are allowed).  The words are
 * the nodes of the paper's graph (Section 3 encoding; Section 5 caps the
 * frequency-sorted list at n).  `flags` may hold NW_DEVICE_PTRS.  The
 * scoring is fixed for the dictionary's lifetime.  On the device the words
 * are sorted stably by length into buckets and encoded for the kernels. */
nw_status nw_load_dictionary(nw_ctx *ctx, const uint8_t *codes, const uint32_t *offsets, uint32_t n,
                             uint32_t alphabet, const nw_scoring *scoring, uint32_t flags,
                             nw_dict **out);

/* The same with Algorithm 1's similarity read from a full matrix (Section 2;
 * Section 6 proposes per-phoneme coefficients): sim[a * alphabet + b] for
 * codes a, b < alphabet <= 64, symmetric, |values| <= 1024, and a linear gap
 * `gap`.  Every all-pairs call, nw_score_pairs, nw_query and the proposal
 * path score such a dictionary with the matrix; the no-allocation variant,
 * the query server and batches take match / mismatch dictionaries only
 * (NW_EINVAL).  The kernels look each cell's term up in a 64 x 64 table of
 * max(sim - 2 * gap, 0) in shared memory; NW_ERANGE if
 * 40 * max(sim - 2 * gap) exceeds 32767.  Histogram bins and the int8 range
 * check use the bounds of match = max(sim), mismatch = min(sim). */
nw_status nw_load_dictionary_sim(nw_ctx *ctx, const uint8_t *codes, const uint32_t *offsets, uint32_t n,
                                 uint32_t alphabet, const int32_t *sim, int32_t gap, uint32_t flags,
                                 nw_dict **out);

/* Fills `out` with facts about the dictionary. */
nw_status nw_dict_info_get(const nw_dict *dict, nw_dict_info *out);

/* Frees a dictionary (NULL is ignored). */
void nw_dict_free(nw_dict *dict);

/* Scores every pair i < j of the dictionary and writes the int8 score of
 * (i, j) at out[S(i-1) + (j - i - 1)], S(i-1) = i(2n - i - 1)/2: the paper's
 * row-major traversal of the upper triangle, (0,1), (0,2), ..., (n-2, n-1),
 * one signed byte per edge (Section 4.1; offsets as in Section 4.2).  `out`
 * holds n(n-1)/2 bytes.  NW_ERANGE if a score of this dictionary can fall
 * outside [-128, 127]. */
nw_status nw_all_pairs_matrix(nw_dict *dict, int8_t *out, uint32_t flags);

/* The same int8 row-major upper triangle for dictionaries whose matrix does
 * not fit in device memory (Section 5's 107,000-word limit, and its proposal
 * to copy intermediate results back and continue): the n(n-1)/2 entries are
 * produced in consecutive chunks of at most chunk_bytes through one device
 * buffer of that size and copied into the host buffer `out` chunk by chunk.
 * Every chunk rescores all pairs and keeps its own entries, so the work grows
 * with the number of chunks.  Host `out` only (NW_DEVICE_PTRS is refused when
 * chunking is needed); chunk_bytes >= n(n-1)/2 is nw_all_pairs_matrix. */
nw_status nw_all_pairs_matrix_chunked(nw_dict *dict, int8_t *out, uint64_t chunk_bytes, uint32_t flags);

/* Scores every pair i < j once and reduces on the device to, for every word,
 * its k best neighbours over all other words (higher score first, lower
 * original index first on equal scores) -- the per-word ego-network lists of
 * Section 5 -- plus the histogram of all n(n-1)/2 scores (Section 5's
 * edge-weight histogram).
 *   nbr_idx[i*k + r], nbr_score[i*k + r]: rank r of word i (n*k entries each).
 *   hist: NULL, or nbins int64 counts; hist[b] counts pairs scoring
 *         *hist_lo + b.  nbins must be >= nw_dict_info.nbins (else NW_ERANGE).
 *   hist_lo: receives the score of bin 0 (may be NULL when hist is NULL).
 * k in [1, NW_MAX_K].  NW_EINVAL if n < 2.
 * With NW_RANK_NORMALISED in `flags` the lists hold the k best neighbours by
 * the length-normalised weight s / max(len_i, len_j) of Section 5 (two empty
 * words: s / 1), compared exactly as fractions; equal weights rank the lower
 * original index first.  nbr_score still receives the raw score s (the
 * paper's displayed weight is 100 * s / max(len_i, len_j)) and the histogram
 * still counts raw scores.  NW_ERANGE if the distinct weights and the index
 * bits of n do not fit 32-bit list keys (for match 1, mismatch -1, gap -1 and
 * words of up to 40 symbols there are under 1,000 weights, so any n up to
 * 2^20 fits).  The flag is accepted by this call only: the shard variant,
 * the no-allocation variant, queries and batches give NW_EINVAL. */
nw_status nw_all_pairs_topk(nw_dict *dict, uint32_t k, uint32_t *nbr_idx, int16_t *nbr_score,
                            int64_t *hist, int32_t *hist_lo, uint32_t nbins, uint32_t flags);

/* The same reduction over shard `shard` of `nshards` disjoint parts of the
 * pair set (every unordered pair belongs to exactly one shard).  The lists
 * hold each word's k best neighbours among the pairs of that shard and the
 * histogram counts that shard's pairs; nw_topk_merge combines the lists of
 * all shards into the full result and histograms add. */
nw_status nw_all_pairs_topk_shard(nw_dict *dict, uint32_t shard, uint32_t nshards, uint32_t k,
                                  uint32_t *nbr_idx, int16_t *nbr_score, int64_t *hist,
                                  int32_t *hist_lo, uint32_t nbins, uint32_t flags);

/* Host-only: merges `nparts` partial neighbour lists of n words (each n*k,
 * ranked as above, missing entries UINT32_MAX / INT16_MIN) into the k best of
 * their union per word, in the same order.  Entries with the same index in
 * several parts must carry the same score; they are kept once.  Host
 * pointers; no GPU is used.  At most 64 parts. */
nw_status nw_topk_merge(uint32_t n, uint32_t k, uint32_t nparts, const uint32_t *const *idx_parts,
                        const int16_t *const *score_parts, uint32_t *idx_out, int16_t *score_out);

/* The same merge on the context's device, for the exchange step of a sharded
 * run after an all-gather: idx_parts / score_parts hold the nparts partial
 * lists one after another (part p of word w at p*n*k + w*k; each list ranked,
 * missing entries UINT32_MAX / INT16_MIN at its end), device pointers; the
 * merged lists go to idx_out / score_out (device, n*k).  Every word is merged
 * by the same k-way merge as nw_topk_merge.  1 <= nparts <= 64; NW_EINVAL
 * otherwise.  Synchronous on the context's stream. */
nw_status nw_topk_merge_device(nw_ctx *ctx, uint32_t n, uint32_t k, uint32_t nparts, const uint32_t *idx_parts,
                               const int16_t *score_parts, uint32_t *idx_out, int16_t *score_out);

/* Scores m explicit pairs (i[p], j[p]) of dictionary words (original indices,
 * i == j allowed) into out[p] (int16).  Each score is Algorithm 1's
 * bottom-right cell for the two words. */
nw_status nw_score_pairs(nw_dict *dict, const uint32_t *i, const uint32_t *j, size_t m, int16_t *out,
                         uint32_t flags);

/* Scores nq query words (CSR as in nw_load_dictionary, codes < the
 * dictionary's alphabet) against every dictionary word and returns each
 * query's k best dictionary neighbours (nbr_idx/nbr_score: nq*k entries,
 * ranked as in nw_all_pairs_topk; a query is not a dictionary word, so no
 * dictionary word is excluded).  This is the "find phonetically similar
 * words" use of Section 6.  flags: NW_DEVICE_PTRS, NW_ASYNC. */
nw_status nw_query(nw_dict *dict, const uint8_t *qcodes, const uint32_t *qoffsets, uint32_t nq,
                   uint32_t k, uint32_t *nbr_idx, int16_t *nbr_score, uint32_t flags);

/* ---- batches of independent dictionaries and query sets ----
 *
 * Many dictionaries of uneven size, length range, alphabet and scoring (each
 * the paper's problem on its own word list, Sections 4-5) reduced to per-word
 * top-k lists in one CUDA-graph launch.  Each dictionary may bring a query
 * set of its own size and lengths (Section 6's search for similar-sounding
 * words, nw_query), answered in the same launch.  nw_batch_create loads every
 * dictionary and query set, plans all their pairs together (one alignment
 * launch per longer length covering every dictionary and query set),
 * optionally autotunes the tile shape (A words per task) of each launch by
 * timing candidates on the batch itself, and captures the whole reduction --
 * list resets, alignment launches, list finalisation -- into a CUDA graph.
 * nw_batch_run / nw_batch_run_queries replay the graph and copy the lists
 * out.  Results equal nw_all_pairs_topk run on each dictionary alone and
 * nw_query run on each query set alone.  The batch uses the context's stream
 * and memory budget; the context must outlive it. */
typedef struct nw_batch nw_batch;

typedef struct {
    const uint8_t *codes;      /* CSR words as in nw_load_dictionary */
    const uint32_t *offsets;
    uint32_t n;
    uint32_t alphabet;
    nw_scoring scoring;
    /* optional query set against this dictionary (nq = 0: none), CSR as in
     * nw_query; copied at creation like the dictionary */
    const uint8_t *qcodes;
    const uint32_t *qoffsets;
    uint32_t nq;
    uint32_t queries_only;     /* nonzero: only the query set is answered; the
                                * dictionary's own lists are not computed */
} nw_batch_dict;

/* nw_batch_create flag: time tile-shape candidates per launch.  Per longer
 * length, the A words per task are chosen from {64, 128, 256}, then the
 * resident blocks per SM from {2, 3, as many as fit} at that size, by timing
 * whole launches on the batch.  (A task's B chunk is 64 words: two words per
 * lane in the kernel's int16x2 registers, fixed at compile time.)  The
 * choices are cached for the life of the process, keyed by the device's SM
 * count, k, and every dictionary's and query set's length histogram, scoring
 * and flags: a batch of the same shape is not timed again (tune_cached = 1). */
#define NW_BATCH_AUTOTUNE 0x10u

typedef struct {
    uint32_t ndicts;
    uint32_t launches;                          /* alignment launches in the graph */
    uint64_t pairs, cells;                      /* over all dictionaries and query sets */
    double tune_ms;                             /* time spent autotuning */
    uint32_t words_per_task[NW_MAX_WORD_LEN + 1]; /* chosen A words per task by longer length (0: none) */
    uint32_t query_words;                       /* words of all query sets */
    uint64_t query_pairs, query_cells;          /* the part of pairs / cells from query sets */
    uint32_t blocks_per_sm[NW_MAX_WORD_LEN + 1]; /* chosen resident blocks per SM by longer length (0: as many as fit) */
    uint32_t tune_cached;                       /* 1: the tile shapes came from the autotuner's cache */
} nw_batch_info;

/* flags: NW_DEVICE_PTRS (the dictionaries' and query sets' buffers are
 * device pointers), NW_BATCH_AUTOTUNE.  k in [1, NW_MAX_K].  Errors as
 * nw_load_dictionary and nw_query: NW_EINVAL for a code >= the dictionary's
 * alphabet (query codes included) or a null query array with nq > 0,
 * NW_ERANGE when a dictionary's or query set's scores do not fit the list
 * keys. */
nw_status nw_batch_create(nw_ctx *ctx, const nw_batch_dict *dicts, uint32_t ndicts, uint32_t k, uint32_t flags,
                          nw_batch **out);

/* Runs the graph.  nbr_idx[d] / nbr_score[d] receive dictionary d's n*k
 * lists (ranked as nw_all_pairs_topk); host buffers, or device buffers with
 * NW_DEVICE_PTRS.  Entries of queries_only dictionaries are not read (may be
 * NULL).  Query lists are computed but not copied out. */
nw_status nw_batch_run(nw_batch *batch, uint32_t *const *nbr_idx, int16_t *const *nbr_score, uint32_t flags);

/* nw_batch_run that also copies dictionary d's query lists, nq*k each and
 * ranked as nw_query, to qnbr_idx[d] / qnbr_score[d] (entries of dictionaries
 * without queries are not read).  Same buffer convention and flags. */
nw_status nw_batch_run_queries(nw_batch *batch, uint32_t *const *nbr_idx, int16_t *const *nbr_score,
                               uint32_t *const *qnbr_idx, int16_t *const *qnbr_score, uint32_t flags);

nw_status nw_batch_info_get(const nw_batch *batch, nw_batch_info *out);

void nw_batch_free(nw_batch *batch);

/* ---- serving: continuous batching of query requests ----
 *
 * A query service over one device-resident dictionary (Section 6's finding of
 * similar-sounding words, run as a service).  Requests (each a CSR batch of
 * query words) are queued by nw_server_submit from any thread.  A worker
 * thread packs queued requests into GPU batches of at most max_batch_queries
 * words and runs each batch on its own stream, with up to max_inflight
 * batches on the device at once: requests that arrive while others run are
 * admitted as soon as a batch slot frees.  Every slot's device buffers are
 * allocated at creation and counted against mem_budget_bytes, which caps the
 * number of slots (admission by memory).  Results are exact and do not depend
 * on which requests share a batch: each query's k best dictionary neighbours,
 * as nw_query returns them.  The dictionary must outlive the server. */
typedef struct nw_server nw_server;

typedef struct {
    uint32_t k;                  /* neighbours per query, 1..NW_MAX_K */
    uint32_t max_batch_queries;  /* words per GPU batch; also the largest request */
    uint32_t max_inflight;       /* batches on the GPU at once (one stream each) */
    uint32_t pad_;
    size_t mem_budget_bytes;     /* device memory for the slots (0 = no cap) */
} nw_server_config;

typedef struct {
    double submit_s, start_s, done_s; /* steady-clock seconds: queued, batch launched, results ready */
    uint32_t nq;                      /* queries of the request */
    uint32_t batch_queries;           /* queries in the batch that carried it */
    uint32_t batch_requests;          /* requests in that batch */
    uint32_t inflight_at_start;       /* batches already on the GPU when it launched */
} nw_request_info;

/* Creates a server for `dict` on the dictionary's device.  NW_ENOMEM if not
 * even one batch slot fits the budget. */
nw_status nw_server_create(nw_dict *dict, const nw_server_config *cfg, nw_server **out);

/* Queues a request of nq host query words (CSR as in nw_load_dictionary;
 * codes < the dictionary's alphabet; 1 <= nq <= max_batch_queries).  The
 * words are copied; *request_id identifies the request. */
nw_status nw_server_submit(nw_server *srv, const uint8_t *qcodes, const uint32_t *qoffsets, uint32_t nq,
                           uint64_t *request_id);

/* Waits up to timeout_ms (< 0: forever) for a request.  On completion copies
 * its nq*k results to host nbr_idx/nbr_score (ranked as nw_query), fills
 * *info (may be NULL), forgets the request and returns its status.  Returns
 * NW_EBUSY if it is still pending, NW_EINVAL for an unknown id. */
nw_status nw_server_wait(nw_server *srv, uint64_t request_id, int timeout_ms, uint32_t *nbr_idx,
                         int16_t *nbr_score, nw_request_info *info);

/* Message for the last failure of a server call or batch ("" if none); with
 * srv == NULL, the message of the last failed nw_server_create on this thread. */
const char *nw_server_last_error(const nw_server *srv);

/* Stops the worker after the batches on the GPU finish, fails queued
 * requests and frees the server. */
void nw_server_destroy(nw_server *srv);

/* ---- variant for callers that cannot allocate device memory ----
 *
 * No counterpart in the paper.  Some callers cannot allocate device memory
 * at the time they run this reduction: code that runs inside a stream
 * capture or with allocation locked down, a real-time loop that must not
 * reach the allocator (cudaMalloc/cudaFree synchronise the device), or a host
 * that has handed all free memory to a pool it manages.  This entry point
 * computes exactly what nw_all_pairs_topk computes for the whole pair set,
 * but takes every scratch buffer (neighbour-list slots, thresholds, task
 * counters, histogram accumulators, error flag) from one fixed static device
 * array of NW_NOALLOC_SCRATCH_BYTES compiled into the library, and calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *   - Outputs must be device pointers: `flags` must contain NW_DEVICE_PTRS
 *     (NW_EINVAL otherwise); hist_lo is a host pointer (may be NULL).
 *   - Scratch needed: 2 KiB + 4*n + 4*n*k + 8*nbins bytes, each part rounded
 *     up to 256 bytes; a dictionary/k that needs more than the array gives
 *     NW_ERANGE and writes nothing (k = 10 allows n up to about 760,000).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture on the device.
 *   - The array is shared by every call in the process and keeps the last
 *     call's contents; each call clears what must start at zero.  Calls whose
 *     GPU work overlaps (other contexts or streams on the same device) race on
 *     the array and give wrong results: serialise them.
 *   - With NW_ASYNC the call returns before its kernels finish, so it cannot
 *     report a device-side failure (a bound that ran out, a score outside the
 *     histogram) itself.  Such a failure is kept in the array and the next
 *     synchronous call of this entry point on the same device reports it
 *     (NW_ETIMEOUT / NW_ERANGE / NW_EINVAL, message naming the earlier
 *     NW_ASYNC call) after computing its own, valid, outputs; then it clears
 *     it.  An NW_ASYNC call never clears it.
 *   - The array occupies device memory on every GPU that loads the library
 *     until the process exits. */
#define NW_NOALLOC_SCRATCH_BYTES (32u << 20)
nw_status nw_all_pairs_topk_noalloc(nw_dict *dict, uint32_t k, uint32_t *nbr_idx, int16_t *nbr_score,
                                    int64_t *hist, int32_t *hist_lo, uint32_t nbins, uint32_t flags);

/* ---- measurement and testing helpers (no counterpart in the paper) ---- */

/* Issue rates of the integer instructions the alignment kernel is built from,
 * measured on the context's device by a throughput microbenchmark over all
 * SMs: dependent chains with 8-way instruction-level parallelism, enough warps
 * to fill every SM, repeated for `ms_target` milliseconds of device time.
 * Rates are per second for the whole GPU, counting one 32-bit instruction per
 * thread as one operation (a packed 16x2 instruction is one operation). */
typedef struct {
    double viaddmax_s16x2;  /* __viaddmax_s16x2 */
    double vimax3_s16x2;    /* __vimax3_s16x2 */
    double vimax_s16x2_relu;/* __vimax_s16x2_relu */
    double iadd3;           /* three-input 32-bit add */
    double lop3;            /* three-input 32-bit logic op */
    double nw_cell_mix;     /* the alignment kernel's per-cell instruction mix, in packed cells/s */
    double sm_clock_mhz;    /* clock64 cycles per microsecond of event time, averaged over the
                             * benchmarks; on a GB300 this reads well below the SM clock that
                             * nvidia-smi reports under the same load, so issue widths are best
                             * derived from the rates and nvidia-smi's clock */
    uint32_t sm_count;
    uint32_t pad_;
} nw_int_rates;

nw_status nw_measure_int_rates(nw_ctx *ctx, double ms_target, nw_int_rates *out);

/* Host-only: the pairs the all-pairs kernels of a dictionary with these word
 * lengths would score for shard `shard` of `nshards`, as original-index pairs
 * (a[p], b[p]), in task order.  Writes at most `cap` pairs and sets *count to
 * the total.  Runs the same planner and task-to-pair mapping as the kernels,
 * on the CPU, so tests can check that every unordered pair is covered exactly
 * once. */
nw_status nw_debug_enumerate_pairs(const uint32_t *lengths, uint32_t n, uint32_t shard,
                                   uint32_t nshards, uint32_t *a, uint32_t *b, uint64_t cap,
                                   uint64_t *count);

/* Host-only: the (query, dictionary word) pairs that nw_query's kernels
 * would score for query words of lengths q_lengths[0..nq) against dictionary
 * words of lengths d_lengths[0..nd), with at most `ta` A words per task (0 =
 * the default; a launch with few tasks takes smaller chunks, down to 32
 * words, as nw_query plans it), as original-index pairs (q[p], d[p]).
 * Writes at most `cap` pairs and sets *count to the total.  Runs the same
 * query planner and task-to-pair mapping as the kernels, on the CPU, so tests
 * can check that every (query, word) pair is covered exactly once. */
nw_status nw_debug_enumerate_query_pairs(const uint32_t *q_lengths, uint32_t nq, const uint32_t *d_lengths,
                                         uint32_t nd, uint32_t ta, uint32_t *q, uint32_t *d, uint64_t cap,
                                         uint64_t *count);

/* Host-only: the tables behind NW_RANK_NORMALISED for scores [lo, hi].
 * *nranks receives the number of distinct weights s/m (rank 0 = smallest);
 * when it is <= cap_ranks, also writes
 *   rank[(s - lo) * (NW_MAX_WORD_LEN + 1) + m]: rank of s/m for longer length
 *       m (m = 0: s/1) where s is reachable for m, else 0;
 *   smin[r * (NW_MAX_WORD_LEN + 1) + m]: smallest reachable s whose s/m has
 *       rank >= r, else INT16_MAX;
 *   frac[2r], frac[2r + 1]: rank r's weight in lowest terms.
 * rank holds (hi - lo + 1) * (NW_MAX_WORD_LEN + 1) entries.  NW_EINVAL for
 * lo > hi or null pointers; NW_ERANGE when *nranks > cap_ranks. */
nw_status nw_debug_norm_tables(const nw_scoring *scoring, int32_t lo, int32_t hi, uint16_t *rank,
                               int16_t *smin, int16_t *frac, uint32_t cap_ranks, uint32_t *nranks);

/* Test hook: the `countdown`-th device allocation of the context from now on
 * fails as if the device were out of memory (0 disables).  Host-side only. */
nw_status nw_debug_fail_alloc(nw_ctx *ctx, uint32_t countdown);

/* Test hook for the device-side bounds (failure detection without a GPU
 * fault).  Later calls on the context use:
 *   insert_iters  >= 0: neighbour-list insertions of the alignment kernels
 *                 give up after this many compare-and-swap rounds (0: at the
 *                 first offer) and the call returns NW_ETIMEOUT; < 0 restores
 *                 the kernel's own bound (2^20 rounds);
 *   wait_cycles   >= 0: every pipeline wait of the candidate kernel
 *                 (nw_dot_topk, nw_dot_topk_cross, the proposal calls) gives
 *                 up after this many SM clock cycles; < 0 restores its own
 *                 bound (2e9 cycles, about a second);
 *   withhold_tile != UINT32_MAX: the candidate kernel's producer never issues
 *                 the bulk copy of this column tile (of 128 columns; the
 *                 tile's index in the CTA's sweep order), so every
 *                 wait for it runs out with no copy in flight; the kernel
 *                 still waits (bounded) for the copies it did issue before it
 *                 exits.  The call returns NW_ETIMEOUT.
 * The context stays usable: a later call with the defaults restored is
 * correct.  Host-side only; NW_EINVAL for a null context. */
nw_status nw_debug_set_bounds(nw_ctx *ctx, int32_t insert_iters, int64_t wait_cycles, uint32_t withhold_tile);

#ifdef __cplusplus
}
#endif

#endif /* NW_H */
