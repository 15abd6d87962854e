/*
 * swgb -- Smith-Waterman protein database search on one NVIDIA GB300 (sm_103a).
 *
 * C ABI of libswgb.so.  Plain pointers and sizes only.
 *
 * What is computed (paper Section 2, Eqs. sw2-sw4): for a query S1 of length m and a
 * database sequence S2 of length n,
 *     H[i][j] = max{0, H[i-1][j-1] + SM(S1[i], S2[j]), E[i][j], F[i][j]}
 *     E[i][j] = max{H[i][j-1] - Goe, E[i][j-1] - Ge}
 *     F[i][j] = max{H[i-1][j] - Goe, F[i-1][j] - Ge}
 * with H, E, F = 0 on row 0 and column 0; the score is max over i, j of H[i][j] (0 if m or
 * n is 0).  One score per database sequence, one query against the whole database: the
 * paper's inter-task database search (Sections 1 and 4).
 *
 * Gap costs: Goe = gap_open, Ge = gap_extend.  A gap of length k costs
 * gap_open + (k - 1) * gap_extend (when gap_extend <= gap_open; otherwise Eqs. sw3/sw4
 * charge each continuing position min(gap_open, gap_extend)).  The paper's own setting
 * "open 10, extend 2" with Goe = open + extend is gap_open = 12, gap_extend = 2.
 *
 * Conventions shared by every call:
 *  - Residues are codes in [0, alphabet_size), alphabet_size <= 32.  A code outside that
 *    range is SW_ERR_CODE.
 *  - The matrix is alphabet_size x alphabet_size int8, row-major, query letter first:
 *    SM(a, b) = matrix[a * alphabet_size + b].
 *  - gap_open >= 0, gap_extend >= 0, both <= 1,000,000.  Scores are int32; SW_ERR_ARG if
 *    min(m, n) * max(SM) could exceed INT32_MAX.
 *  - Zero-length queries and sequences are allowed and score 0.
 *  - On a non-OK status no output is defined; sw_last_error() says why (thread-local).
 *  - Host input buffers are borrowed for the duration of the call only.
 *  - Calls on one database handle are serialised internally.
 *
 * Environment switches (experiments; the defaults are the measured best): SWGB_MQ=0 (no
 * two-queries-per-register kernel), SWGB_VARIANT=v (force an inter-task variant, read at
 * load), SWGB_GROUP_SPLIT=s (groups [0, s) on the inter-task kernel, the rest on the int32
 * intra-task kernel), SWGB_INTRA_BLOCK=0 (per-warp int32 kernel, read at load),
 * SWGB_INTRA_BLOCKS_PER_SM=n, SWGB_SCORE_PROFILE=1 (score-profile single-query kernel,
 * Section 4.3), SWGB_WAVE=0 (int32 instead of the packed int16x2 wavefront kernel for long
 * subjects), SWGB_WAVE_ROWS=8|12|16 (its rows per lane), SWGB_PAIR=0 (int32 instead of the
 * packed two-subject wavefront for the routed groups of one query), SWGB_PAIR_HALF=1|auto (its
 * bulk on two 16-lane wavefronts per warp whenever they fit, or where the plan's cost model
 * prefers them; default: 32-lane wavefronts only), SWGB_PAIR_HALF_FROM=i (16-lane items from
 * slot pair i on), SWGB_LONG_PAIRS=n,
 * SWGB_LONG_BLOCKS=n (its first phase), SWGB_GRAPHS=0 (no CUDA-graph capture).  Scores do not
 * depend on them.
 */
#ifndef SWGB_H
#define SWGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sw_db sw_db;          /* device-resident database, owned by the library */
typedef struct sw_server sw_server;  /* continuous-batching search server */

typedef enum {
    SW_OK = 0,
    SW_ERR_ARG = -1,      /* invalid argument (null pointer, bad size, bad gap cost) */
    SW_ERR_CODE = -2,     /* a residue code >= alphabet_size */
    SW_ERR_OOM = -3,      /* device or host allocation failed */
    SW_ERR_CUDA = -4,     /* a CUDA call failed (message in sw_last_error) */
    SW_ERR_TIMEOUT = -5,  /* a bounded wait ran out */
    SW_ERR_BUSY = -6,     /* server: no admission capacity for this request now */
    SW_ERR_STATE = -7     /* call not valid in the object's current state */
} sw_status;

/* Options for sw_db_load_ex.  Zero fields take the defaults. */
typedef struct {
    int32_t device;        /* CUDA device ordinal (default: the current device) */
    int32_t long_cutoff;   /* sequences longer than this go to the intra-task kernel
                              (default 3072; must be a multiple of 8) */
    int32_t flag_cap;      /* capacity of the list of saturated int16 lanes (default 2^20);
                              when more lanes saturate, the rescore sweeps every score */
    int32_t placement;     /* SW_PLACE_DEVICE (default): the database is copied to HBM.
                              SW_PLACE_HOST: the database stays in pinned host memory mapped
                              into the device address space, and the kernels stream it over
                              the CPU-GPU link while they compute -- for databases larger than
                              HBM (the paper's future work, Section 6). */
    int32_t reserved[4];
} sw_db_options;

#define SW_PLACE_DEVICE 0
#define SW_PLACE_HOST 1

/* Per-call measurements of the last search on a handle (CUDA events on the launch stream). */
typedef struct {
    float inter_ms;        /* inter-task int16x2 kernel */
    float intra_ms;        /* intra-task int32 kernel (long subjects, routed groups) */
    float rescore_ms;      /* int32 rescore of saturated lanes */
    float total_ms;        /* first to last launch of the search */
    int64_t cells;         /* sum over queries of m * (database residues) */
    int64_t inter_cells;   /* cells the inter-task kernel covered (real residues) */
    int64_t flagged;       /* lanes that reached the int16 threshold and were rescored */
    int64_t launches;      /* kernels launched by the search */
    int32_t inter_grid;    /* persistent grid of the inter-task kernel (blocks) */
    int32_t inter_block;   /* threads per block of the inter-task kernel */
    int32_t graph_replay;  /* 1 if the launch sequence was a replayed CUDA graph */
    int32_t variant;       /* inter-task kernel variant used (see sw_db_tune) */
    int32_t multi_query;   /* 1 if two queries shared each register (two or more queries) */
    int32_t score_profile; /* 1 if the single-query inter-task kernel used a score profile
                              (Section 4.3; environment SWGB_SCORE_PROFILE=1) */
    int32_t intra_packed;  /* intra-task work on the packed int16x2 wavefront kernel instead
                              of int32: 1 = two queries per register (long subjects of a
                              batch), 2 = two subjects per register (routed groups of a
                              one-query search), 0 = int32 only */
    int32_t wave_lanes;    /* lanes per wavefront of the packed kernel: 32, or 16 when some
                              warps ran two 16-lane wavefronts (the shorter pairs of
                              intra_packed = 2); 0 without a packed intra-task launch */
} sw_stats;

/* ---------------------------------------------------------------- database ------------ */

/* Preprocessing stage (paper Section 4: sort by length ascending, pad with a dummy symbol,
 * group by lane count).  Copies `residues[0 .. offsets[num_seqs])`, sequence k being
 * residues[offsets[k] .. offsets[k+1]), to the device in a length-sorted, 64-sequence
 * interleaved layout plus a plain copy.  offsets must start at 0 and be non-decreasing.
 * The caller keeps its buffers; the handle is freed with sw_db_free.  SW_ERR_ARG on a bad
 * size or offset, SW_ERR_CODE on a residue code >= alphabet_size, SW_ERR_OOM when device
 * memory runs out; *out is NULL on any error. */
sw_status sw_db_load(const uint8_t *residues, const int64_t *offsets, int64_t num_seqs,
                     int32_t alphabet_size, sw_db **out);
/* sw_db_load with options (Section 4 preprocessing; the placement option serves the paper's
 * future-work case of a database larger than memory, Section 6). */
sw_status sw_db_load_ex(const uint8_t *residues, const int64_t *offsets, int64_t num_seqs,
                        int32_t alphabet_size, const sw_db_options *opts, sw_db **out);
/* Releases a database from sw_db_load[_ex] after its searches finish (NULL is a no-op).
 * Sizes of the database of Section 4's preprocessing stage (-1 for a NULL handle). */
void sw_db_free(sw_db *db);
int64_t sw_db_num_seqs(const sw_db *db);
int64_t sw_db_num_residues(const sw_db *db);

/* ---------------------------------------------------------------- search -------------- */

/* SW stage (paper Section 4) for one query: scores[k] = best local score of the query
 * against database sequence k (original order).  Host query, host matrix, host output
 * buffer of num_seqs int32.  Synchronous. */
sw_status sw_search(const sw_db *db, const uint8_t *query, int32_t query_len,
                    const int8_t *matrix, int32_t gap_open, int32_t gap_extend,
                    int32_t *scores);

/* SW stage (paper Section 4) for several queries in one persistent launch, work items drawn
 * dynamically by idle blocks (the dynamic distribution of Section 4.1).  queries[q] has
 * query_lens[q] residues (host).  scores is a host buffer of num_queries * num_seqs int32,
 * row q = query q, original database order.  Synchronous.  Errors as sw_search. */
sw_status sw_search_batch(const sw_db *db, const uint8_t *const *queries,
                          const int32_t *query_lens, int32_t num_queries,
                          const int8_t *matrix, int32_t gap_open, int32_t gap_extend,
                          int32_t *scores);

/* SW stage (paper Section 4; dynamic distribution of work, Section 4.1), device-resident
 * variant for callers that hold device memory (e.g. PyTorch tensors).
 * d_queries: device buffer of concatenated query residues; query_offsets: HOST array of
 * num_queries + 1 int64 offsets into it.  matrix: host.  d_scores: device buffer of
 * num_queries * num_seqs int32 (row q = query q, original database order), owned by the
 * caller.  Work is enqueued on `stream` (a cudaStream_t, NULL = the legacy default stream);
 * the call returns without waiting for it.  Repeated calls with the same shapes and pointers
 * replay a captured CUDA graph.  Argument errors are returned at once; a query residue code
 * >= alphabet_size is detected on the device and returned as SW_ERR_CODE by the next
 * sw_get_stats on the handle. */
sw_status sw_search_batch_device(const sw_db *db, const uint8_t *d_queries,
                                 const int64_t *query_offsets, int32_t num_queries,
                                 const int8_t *matrix, int32_t gap_open, int32_t gap_extend,
                                 int32_t *d_scores, void *stream);
/* The same call under the name of the asynchronous device-pointer search (Section 4 SW
 * stage, Section 4.1 dynamic distribution): identical arguments, behaviour and errors. */
sw_status sw_search_async(const sw_db *db, const uint8_t *d_queries,
                          const int64_t *query_offsets, int32_t num_queries,
                          const int8_t *matrix, int32_t gap_open, int32_t gap_extend,
                          int32_t *d_scores, void *stream);

/* Autotuner.  The inter-task kernel comes in variants (query rows per strip x warps per
 * block, e.g. 32x4, 64x4, 32x8, 64x8: registers vs. occupancy vs. per-column overhead).
 * sw_db_tune runs the given probe queries (host) against the whole database once per variant
 * (after one warm-up run), times the inter-task kernel with CUDA events, and makes the fastest
 * variant the one every later search on `db` uses.  If `cache_path` is non-NULL the choice is
 * looked up there first (key: device name, SM count, alphabet size, database shape, probe
 * length class) and stored there after tuning; with `force` the cache is ignored on lookup.
 * The counterpart of the paper's tuning of thread counts and instruction sets by measurement
 * (Section 5.2), done here automatically per database.  Errors as sw_search; a cache file
 * that cannot be read or written is ignored. */
typedef struct {
    int32_t variant;             /* chosen variant index */
    int32_t rows_per_strip;      /* its query rows per strip */
    int32_t warps_per_block;     /* its warps per block */
    int32_t from_cache;          /* 1 if taken from the cache without timing */
    int32_t num_variants;
    float gcups[8];              /* inter-task kernel GCUPS per variant (0 = not run) */
} sw_tune_result;
sw_status sw_db_tune(sw_db *db, const uint8_t *const *queries, const int32_t *query_lens,
                     int32_t num_queries, const int8_t *matrix, int32_t gap_open,
                     int32_t gap_extend, const char *cache_path, int32_t force,
                     sw_tune_result *out);

/* Selects an inter-task kernel variant directly (-1 restores the default); the manual form
 * of the Section 5.2 tuning.  SW_ERR_ARG for an unknown variant. */
sw_status sw_db_set_variant(sw_db *db, int32_t variant);

/* Measurements of the last completed search on `db` (synchronises the handle's stream):
 * kernel times and the cells of Eq. gcups (Section 5).  Returns the SW_ERR_CODE that a
 * device-side residue check of the last search found. */
sw_status sw_get_stats(const sw_db *db, sw_stats *out);

/* ---------------------------------------------------------------- sorting stage ------- */

/* Sorting stage (paper Section 4, step 3: alignment scores sorted in descending order), as a
 * top-k: for each of num_queries score rows on the device (row q = d_scores + q * num_seqs,
 * scores >= 0 as the searches return them), the k best database sequences in descending
 * score order, equal scores by ascending sequence index.  Outputs on the device:
 * d_top_scores[q * k + r] and d_top_ids[q * k + r], r = 0 .. k-1.  k <= SW_TOPK_MAX and
 * k <= num_seqs.  Enqueued on `stream` (NULL = legacy default stream). */
#define SW_TOPK_MAX 4096
sw_status sw_topk(const int32_t *d_scores, int64_t num_seqs, int32_t num_queries, int32_t k,
                  int32_t *d_top_scores, int32_t *d_top_ids, void *stream);

/* ---------------------------------------------------------------- serving ------------- */

/* Continuous-batching search server over a resident database: not in the paper (it searches
 * one query at a time, Section 4; serving is this library's addition).  Requests (one query each) are admitted
 * while a slot is free and their DP state fits the budget; DP state of a request = its query
 * profile ((A+1) x ceil(m/256)*256 int16) plus its score row (num_seqs int32).  The database
 * is cut into `slices` of about equal residue work; a background thread runs "ticks" that scan
 * the slices cyclically.  In a tick every in-flight request aligns against the current slice:
 * one replay of a captured CUDA graph, with two queries per int16x2 register when two or more
 * requests are in flight (split into independent batches when that is needed to keep the GPU
 * busy), followed by the int32 work (long subjects of newly admitted
 * requests, saturated lanes).  A request admitted while others run joins at the next tick and
 * completes after one full cycle of slices; its scores (original order) are then copied to the
 * host.  A request that finds the server idle and nothing pending scans the whole database in
 * one tick when that tick is short against the recent gaps between submissions.  Each score
 * equals the one sw_search returns for the same query.
 * Gap costs must fit the int16 path (gap_open, gap_extend <= 16383). */
typedef struct {
    int32_t max_inflight;        /* requests on the GPU at once (default 32, max 128) */
    int32_t max_query_len;       /* longest accepted query (default 8192) */
    int64_t state_budget_bytes;  /* DP-state bytes of all in-flight requests (default 1 GiB) */
    int32_t slices;              /* database slices of the cyclic scan; a request takes one
                                    tick per slice (default: as many as keep ~8 waves of work
                                    items per tick, at most 16) */
    int32_t max_pending;         /* submitted but not admitted (default 4096) */
    int32_t reserved[6];
} sw_server_options;

typedef struct {
    int64_t submitted, completed, rejected, ticks;
    int32_t in_flight, max_in_flight;
    int64_t joined_while_running; /* admissions while other requests were in flight */
    double latency_p50_ms, latency_p99_ms, latency_mean_ms, latency_max_ms;
    double gcups;                 /* cells of completed requests / (last completion - first submit) */
    int64_t cells;
} sw_server_stats;

sw_status sw_server_create(sw_db *db, const int8_t *matrix, int32_t gap_open, int32_t gap_extend,
                           const sw_server_options *opts, sw_server **out);
/* Serving calls: not in the paper (a request loop on top of its Section 4 search).
 * sw_server_submit copies the query and returns a ticket; SW_ERR_BUSY if max_pending
 * requests are waiting, SW_ERR_ARG / SW_ERR_CODE for a bad query. */
sw_status sw_server_submit(sw_server *srv, const uint8_t *query, int32_t query_len,
                           int64_t *ticket);
/* Not in the paper (serving).  If the request is done, copies its num_seqs scores to
 * `scores`, sets *done = 1 and retires the ticket; otherwise sets *done = 0. */
sw_status sw_server_poll(sw_server *srv, int64_t ticket, int32_t *scores, int32_t *done);
/* Not in the paper (serving).  Waits up to timeout_ms (bounded; SW_ERR_TIMEOUT) for the
 * request, then as sw_server_poll. */
sw_status sw_server_wait(sw_server *srv, int64_t ticket, int32_t *scores, int32_t timeout_ms);
/* Not in the paper (serving).  Counters, latency percentiles and the GCUPS of Eq. gcups
 * over completed requests (reset = 1 clears them). */
sw_status sw_server_get_stats(sw_server *srv, sw_server_stats *out, int32_t reset);
/* Not in the paper (serving).  Stops the loop (in-flight work finishes first) and frees
 * the server. */
void sw_server_destroy(sw_server *srv);

/* ---------------------------------------------------------------- host-side plan ------ */

/* Host-only view of the preprocessing stage (paper Section 4: length sort, grouping, dummy
 * padding), for inspection and tests (no GPU needed).  SW_ERR_ARG / SW_ERR_CODE as
 * sw_db_load.
 * sw_layout_sizes reports the sizes; sw_layout_build fills caller-owned buffers:
 *   group_off[num_groups]   byte offset of each 64-sequence group in `inter`
 *   group_len[num_groups]   padded column count of the group (multiple of 8)
 *   perm[num_groups * 64]   original sequence id of each group slot, -1 for fillers
 *   inter[inter_bytes]      interleaved residues: position j of slot s = 2t + l of group g
 *                           is inter[group_off[g] + (j / 8) * 512 + t * 16 + (j % 8) * 2 + l],
 *                           the dummy code alphabet_size past the end of the sequence
 *   long_ids[num_long]      ids of sequences longer than long_cutoff, longest first
 * Groups are in ascending length order. */
sw_status sw_layout_sizes(const int64_t *offsets, int64_t num_seqs, int32_t long_cutoff,
                          int64_t *num_groups, int64_t *inter_bytes, int64_t *num_long);
sw_status sw_layout_build(const uint8_t *residues, const int64_t *offsets, int64_t num_seqs,
                          int32_t alphabet_size, int32_t long_cutoff, int64_t *group_off,
                          int32_t *group_len, int32_t *perm, uint8_t *inter,
                          int32_t *long_ids);

/* ---------------------------------------------------------------- no device allocation */

/* The paper has no counterpart to this entry point; it exists for callers that cannot let a
 * library allocate device memory at search time.  The other search calls grow a per-database
 * workspace with cudaMalloc when a larger search arrives.  That does not suit a service that
 * overlaps many streams (cudaMalloc/cudaFree may synchronise the whole device), a process
 * whose device memory is already handed out by another allocator (a framework's caching
 * allocator, a pool sized at start-up, a container with a hard limit), or code that must not
 * allocate after initialisation.
 *
 * sw_search_noalloc scores one query against every database sequence, like
 * sw_search_batch_device with num_queries = 1, and calls no allocation routine: all its
 * working memory lives in one fixed array of SW_NOALLOC_SCRATCH_BYTES (about 85 MiB) inside
 * the library's device image.  That array is held on every device where this entry point
 * runs until the process exits.  The first call on a device resolves the array's address
 * there (with that device current); make that first call before any stream capture.
 *   d_query   device buffer of query_len residue codes (each < alphabet_size; an
 *             out-of-range code is scored as 0)
 *   matrix    host, alphabet_size x alphabet_size int8 (read before the call returns;
 *             it reaches the device inside a kernel's parameters, not by a host copy)
 *   d_scores  device buffer of sw_db_num_seqs(db) int32, original database order
 *   stream    cudaStream_t (NULL = legacy default stream); the call only enqueues work.
 * Limits: query_len <= SW_NOALLOC_MAX_QUERY; a database whose groups or sequences are too
 * long for the fixed boundary buffers, or with more than 2^20 groups, is rejected with
 * SW_ERR_ARG.  The boundary buffers bound the number of resident blocks, so large databases
 * search more slowly than with sw_search_batch_device.
 * Every call shares the one array: calls whose work overlaps on the GPU (different streams,
 * or different host threads without ordering) race and give undefined scores.  Serialise
 * them, e.g. on one stream. */
#define SW_NOALLOC_MAX_QUERY 8192
#define SW_NOALLOC_SCRATCH_BYTES 89147904
sw_status sw_search_noalloc(const sw_db *db, const uint8_t *d_query, int32_t query_len,
                            const int8_t *matrix, int32_t gap_open, int32_t gap_extend,
                            int32_t *d_scores, void *stream);

/* ---------------------------------------------------------------- misc ---------------- */

/* Library housekeeping, not in the paper: the message of the last non-OK status on this
 * thread (never NULL), the library version, and the number of kernels this library has
 * launched in this process. */
const char *sw_last_error(void);
const char *sw_version(void);
int64_t sw_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* SWGB_H */
