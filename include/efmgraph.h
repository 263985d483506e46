/*
 * efmgraph.h -- C-ABI of the GB300 flux-balanced pathway library.
 *
 * The library enumerates flux-balanced, elementary pathways of a metabolic
 * network by exhaustive traversal of its AND/OR graph (metabolites are OR
 * nodes, reactions AND nodes; Sec. 2.2, Def. 4-7).  Input: the
 * stoichiometric matrix S (Sec. 2.1) with reversibility and external flags.
 * Output: the set of minimal flux-balanced pathways (Alg. 1 input/output),
 * each reported as its reaction support over split columns.
 *
 * Conventions
 *  - Every function returns 0 on success, a negative EFM_E* code on error
 *    (no partial results are then defined), or for efm_find_pathways /
 *    efm_fetch_results possibly a positive combination of EFM_TRUNCATED,
 *    EFM_CAPPED, EFM_OVERFLOW_DROPPED (completed with warnings).
 *  - Nothing is thrown across this boundary.  Handles are not thread-safe:
 *    use one handle from one host thread at a time.
 *  - All host arrays passed in are copied before the call returns; the
 *    caller keeps ownership.  Device memory is owned by the library and
 *    released by the matching efm_free_*.
 *  - Split columns: reaction j gives column "forward j"; a reversible
 *    reaction also gives the next column "reverse j" (the direction of
 *    Def. 6).  efm_column_map() returns the mapping.
 *  - Supports are bitsets of W = ceil(N / 64) little-endian uint64 words,
 *    column k at bit (k % 64) of word (k / 64).
 */
#ifndef EFMGRAPH_H
#define EFMGRAPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define EFM_OK 0
#define EFM_EINVAL (-1)      /* bad argument or malformed network */
#define EFM_ENOMEM (-2)      /* device or host allocation failed */
#define EFM_ECAPACITY (-3)   /* a device buffer limit was exceeded */
#define EFM_ETIMEOUT (-4)    /* a bounded device-side wait gave up */
#define EFM_ECUDA (-5)       /* a CUDA runtime call failed */
#define EFM_EUNSUPPORTED (-6) /* outside the supported sizes (see limits) */

#define EFM_TRUNCATED 1        /* a level's frontier exceeded max_frontier */
#define EFM_CAPPED 2           /* max_results reached; smallest kept */
#define EFM_OVERFLOW_DROPPED 4 /* some child balances left the int32 range */

/* ---- supported sizes --------------------------------------------------- */
#define EFM_MAX_COLUMNS 4096   /* split columns N (support width 64 words) */
#define EFM_MAX_INTERNAL 1024  /* internal metabolites */
#define EFM_MAX_LEN 64         /* max_len (pathway length in columns) */
#define EFM_MAX_COEF 524287    /* |stoichiometric coefficient| */

typedef struct efm_net efm_net;     /* opaque, library-owned */
typedef struct efm_job efm_job;     /* opaque, library-owned */
typedef struct efm_model efm_model; /* opaque, library-owned */

/* Limits of one traversal (the MAX_LOOP bound of Sec. 3.2 and the length
 * bound L of Alg. 1, plus level-granular budgets). */
typedef struct {
    int32_t max_len;       /* max |U| in split columns, 1..EFM_MAX_LEN */
    int32_t max_secondary; /* max secondary steps per pathway (Def. 10, Eq. 4), >= 0 */
    int64_t max_results;   /* <= 0: no cap; else stop after the level reaching it (EFM_CAPPED) */
    int64_t max_frontier;  /* <= 0: no budget (2^22 states per level); else stop when a level
                              exceeds it (EFM_TRUNCATED); at most 2^31 */
    int32_t first_k;       /* 0: every result; K > 0: exactly the K smallest results in the
                              output order (|U|, then the ascending column list).  Found by
                              traversals with the length cap deepened, P = 1, 2, ... up to
                              max_len, until one holds at least K results (those of size <= P
                              are exactly that run's results), each with an exact branch and
                              bound; a level over max_frontier is split into parts run one after
                              the other; the counters are those of the last run.  The answer is
                              certified unless EFM_TRUNCATED is set.  max_results must be 0
                              (not with the batched call) */
    int32_t proposal;      /* order of a first-K search: EFM_PLAIN (arena order) or
                              EFM_LEARNED (scores of the model passed with the call); the
                              result set is the same either way */
    int32_t variant;       /* EFM_ADDITIVE: flux is only ever added (Eq. 3, Eq. 4);
                              EFM_SUBTRACTIVE: also Eq. 5 -- the acting metabolite may be
                              balanced by taking flux away from a reaction already in the
                              pathway that moves it the same way as its imbalance; a step
                              that leaves that reaction with zero (or negative) flux is
                              discarded (Prop. 3) and counted in zero_flux.  Such a step
                              keeps the support and costs one secondary step.  States then
                              carry their flux vector, so distinct states are distinct
                              (support, flux ray); the network needs internal metabolites
                              + split columns <= EFM_MAX_INTERNAL (else EFM_EUNSUPPORTED),
                              and first_k must be 0.  efm_find_pathways and
                              efm_find_pathways_from only (the batched call is additive). */
    int32_t reserved;      /* must be 0 */
} efm_limits;

#define EFM_PLAIN 0
#define EFM_LEARNED 1
#define EFM_ADDITIVE 0
#define EFM_SUBTRACTIVE 1

/* Counters of one (network, target) traversal; the same definitions as the
 * CPU oracle's.  frontier / frontier_max exclude a truncated level. */
typedef struct {
    int64_t levels;       /* levels executed (level 0 = seeds) */
    int64_t seeds;        /* seed pathways created (INIT) */
    int64_t expansions;   /* children materialised by the AND update (Eq. 3/4) */
    int64_t overflow;     /* children dropped: balance outside int32 */
    int64_t balanced;     /* balanced pathways produced (with multiplicity) */
    int64_t candidates;   /* distinct balanced supports judged */
    int64_t results;      /* supports accepted as elementary (before capping) */
    int64_t pruned;       /* children dropped: support contains a result */
    int64_t frontier;     /* sum over levels of distinct frontier states */
    int64_t frontier_max; /* largest level frontier */
    int64_t status;       /* EFM_TRUNCATED | EFM_CAPPED | EFM_OVERFLOW_DROPPED */
    int64_t zero_flux;    /* EFM_SUBTRACTIVE only: children discarded because a subtractive
                             step (Eq. 5) left a reaction with no positive flux (Prop. 3) */
} efm_counters;

/* Load a network (Alg. 1 "convert S to the MG graph and copy it to the GPU").
 *  n_met, n_rxn          : S is n_met x n_rxn
 *  row_ptr[n_met + 1]    : CSR by metabolite; row_ptr[0] = 0, non-decreasing
 *  col_idx[nnz]          : reaction index in [0, n_rxn), unique within a row
 *  coef[nnz]             : net coefficient S[m][j] (Sec. 2.1), nonzero,
 *                          |coef| <= EFM_MAX_COEF
 *  reversible[n_rxn]     : 1 = reversible (split into two columns)
 *  external[n_met]       : 1 = external metabolite (not balanced, Def. 2)
 *  cuda_stream           : cudaStream_t (0 = legacy default) used by every
 *                          later call on this network and its jobs
 *  out                   : receives the handle
 * Errors: EFM_EINVAL for a malformed CSR, zero or out-of-range
 * coefficients, N > EFM_MAX_COLUMNS or internal > EFM_MAX_INTERNAL;
 * EFM_ENOMEM / EFM_ECUDA on allocation or copy failure. */
int efm_load_network(int32_t n_met, int32_t n_rxn, const int32_t *row_ptr, const int32_t *col_idx,
                     const int32_t *coef, const uint8_t *reversible, const uint8_t *external,
                     uintptr_t cuda_stream, efm_net **out);

/* Split-column count N and support width W of a loaded network. */
int efm_network_shape(const efm_net *net, int32_t *n_columns, int32_t *words_per_set,
                      int32_t *n_internal);

/* Column map: orig_rxn[N] = reaction of each split column, dir[N] = +1
 * forward / -1 reverse.  Either pointer may be NULL. */
int efm_column_map(const efm_net *net, int32_t *orig_rxn, int8_t *dir);

/* Enumerate the pathways of each target (Prop. 1: pathways seeded by the
 * reactions producing the target; -1 = every column).  Runs the level loop
 * of seed -> expand (OR branches, AND update, ballot/popc tests, hash dedup
 * and compaction, superset pruning) -> exact mod-p minimality test on the
 * network's stream and returns when all targets are done.
 *  targets[n_targets]    : metabolite indices in [0, n_met) or -1
 *  limits                : see efm_limits
 *  model                 : NULL, or a proposal model (efm_model_create) when
 *                          limits->proposal is EFM_LEARNED
 *  out                   : receives the job handle (results stay on device
 *                          until fetched or freed)
 * Returns the OR of the warning flags over all targets, or an error. */
int efm_find_pathways(efm_net *net, const int32_t *targets, int32_t n_targets, const efm_limits *limits,
                      const efm_model *model, efm_job **out);

/* The traversal from a seed set R_in (Prop. 1): one starting pathway with
 * flux 1 on each of the given split columns (EF = the sum of their S_int
 * columns, normalised), then the same level loop, limits, pruning and
 * minimality test as efm_find_pathways; the results are the elementary
 * pathways reached from it (each contains R_in).  The starting state sits
 * at level n_columns - 1 (a state's level is |U| - 1 + secondary steps).
 *  columns    host, n_columns distinct split columns (efm_column_map), no
 *             two of the same reaction, 1 <= n_columns <= max_len
 *  limits     as efm_find_pathways (first_k allowed; proposal must be
 *             EFM_PLAIN)
 *  out        one job entry
 * Returns the warning flags or an error (EFM_EINVAL for a bad set). */
int efm_find_pathways_from(efm_net *net, const int32_t *columns, int32_t n_columns, const efm_limits *limits,
                           efm_job **out);

/* Flux-dependent reactions (Def. 11): the DEPTHy pre-pass (Alg. 2).
 * A step from internal metabolite m goes through a split column k that
 * consumes m to an internal metabolite that k produces; steps out of m are
 * ordered by (column, product row) and r is the most steps out of any
 * internal metabolite.  For each internal metabolite i, every walk of at
 * most `depth` steps from i is enumerated as in Alg. 2 (r^depth digit
 * strings, one per thread); a walk that comes back to i tags its leaving
 * column in dep_out and its returning column in dep_in.
 *  depth      1 .. 16, with r^depth <= 2^40 (else EFM_EUNSUPPORTED)
 *  dep_out    host, M_int x words_per_set uint64 bitsets over split
 *  dep_in     columns, one row per internal metabolite (original order)
 *  steps_max  receives r (may be NULL)
 *  kernel_ms  receives the kernel's device time (may be NULL)
 * Synchronous on the network's stream. */
int efm_dependent_reactions(efm_net *net, int32_t depth, uint64_t *dep_out, uint64_t *dep_in, int32_t *steps_max,
                            double *kernel_ms);

/* Exact flux vectors of results (Def. 3).  For a support U whose columns
 * have nullity(S_int[:, U]) = 1, the balanced flux modes on U form one ray;
 * this returns its primitive integer representative (entries with gcd 1),
 * which is positive on every column of U.  Computed on the device, one warp
 * per support, by exact integer elimination of the rows U touches.
 *  supports  host, n x words_per_set uint64 (e.g. rows of efm_fetch_results)
 *  flux      host, n x EFM_FLUX_COLUMNS int64: row r holds the flux of the
 *            support's columns in ascending column order, zero-padded
 *  status    host, n: 1 = exact vector; 0 = an intermediate value left int64
 *            (row zeroed); -1 = not a single positive ray (nullity != 1, no
 *            columns, more than 64 columns, or mixed signs; row zeroed)
 * Synchronous on the network's stream.  Errors: EFM_EINVAL, EFM_ENOMEM,
 * EFM_ECUDA. */
#define EFM_FLUX_COLUMNS 64
int efm_flux_vectors(efm_net *net, const uint64_t *supports, int64_t n, int64_t *flux, int8_t *status);

/* Failure detection, on demand.  Every device-side wait of the library (a
 * hash slot claimed by another warp but not yet published, a bulk copy's
 * mbarrier) polls a bounded number of times; at the bound the kernel sets
 * a timeout bit in its error word and returns, and the call reports
 * EFM_ETIMEOUT.  This call takes that path on purpose: one kernel waits on
 * a device flag that nothing sets, gives up after 2^20 polls (each with a
 * short sleep; about a second in all) and flags the timeout, which
 * the host maps as it maps a traversal's error word.  Nothing faults or
 * hangs, and the network and its stream stay usable afterwards.
 *  polls      receives the number of polls made (may be NULL)
 *  waited_ms  receives the kernel's device time (may be NULL)
 * Returns EFM_ETIMEOUT (the expected outcome), or EFM_EINVAL, EFM_ENOMEM,
 * EFM_ECUDA.  Synchronous on the network's stream. */
int efm_check_bounded_wait(efm_net *net, int64_t *polls, double *waited_ms);

/* Monte-Carlo mode: the paper's own method (Alg. 3 with its random
 * choices, Theorem 1), in the exact integer form of the traversal.  Walk w
 * (0 <= w < n_walks) starts at a random seed column of the target and takes
 * one random valid OR branch per step until its pathway is balanced (its
 * support is then judged once, like the traversal's), has no valid branch
 * (dead end) or leaves the int32 range (overflow).  Random numbers: walk w
 * uses counters 128 w + s, s = 0 for the seed and s >= 1 for step s; the
 * number of counter c is the first output of SplitMix64 started from state
 * seed + c * 0x9E3779B97F4A7C15, reduced modulo the number of choices
 * (seed columns in ascending order; valid branches in ascending column
 * order).  The result set is therefore reproducible and lies inside the
 * exhaustive traversal's result set for the same limits.
 *  limits   max_len and max_secondary as for efm_find_pathways
 *           (max_secondary <= 63); the other fields must be 0
 *  out      one job entry; efm_fetch_results returns the distinct accepted
 *           supports, sorted; counters: seeds = walks started, expansions =
 *           AND updates, balanced / overflow / pruned = walks that ended
 *           balanced / by overflow / at a dead end, levels = the most steps
 *           of one walk, frontier counters 0.
 * Returns the warning flags (EFM_OVERFLOW_DROPPED) or an error. */
int efm_sample_pathways(efm_net *net, int32_t target, const efm_limits *limits, uint64_t seed, int64_t n_walks,
                        efm_job **out);

/* Batched traversal: job i enumerates the pathways of targets[i] in
 * nets[i] (Prop. 1 seeds, the same method and counters as
 * efm_find_pathways), for thousands of uneven networks in ONE persistent
 * kernel launch captured in a CUDA graph.  Each CTA of the launch takes jobs
 * from a device queue and runs a job's whole level loop in its own scratch
 * slice.  An autotuner picks the CTAs per SM and the queue order (input
 * order or largest network first) by timing a sample of the jobs, and caches
 * the choice per (job count, row class, SM count).
 *  nets[n_jobs]     loaded networks (any mix; all on nets[0]'s stream and
 *                   device; at most 256 internal metabolites each, else
 *                   EFM_EUNSUPPORTED before anything is launched)
 *  targets[n_jobs]  target metabolite per job (or -1)
 *  limits           as efm_find_pathways; max_frontier must be > 0 (it sizes
 *                   each CTA's frontier arena); each job uses
 *                   min(max_len, its column count)
 *  model            must be NULL (first-K and proposals are not batched)
 *  out              one job handle with n_jobs entries for efm_fetch_results
 * Per-job device errors (capacity, bounded waits) are reported by
 * efm_fetch_results for that entry.  Per job at most 2^15 distinct balanced
 * supports and 2^13 results. */
int efm_find_pathways_batch(efm_net *const *nets, const int32_t *targets, int32_t n_jobs, const efm_limits *limits,
                            const efm_model *model, efm_job **out);

/* Launch configuration of the batched traversal (no counterpart in the
 * paper, whose runs are single networks). */
typedef struct {
    int32_t ctas_per_sm;     /* persistent CTAs launched per SM, at most what the SM holds; when
                                pinning, 0 = as many as the SM holds */
    int32_t largest_first;   /* 1: the queue runs the networks with the most columns x internal
                                metabolites first; 0: input order */
    int32_t warps_per_job;   /* warps of the CTA that runs one job: 4 or 8 */
    int32_t tile;            /* most parents a warp expands per pass, 1..32 */
    int32_t queue_chunk;     /* queue positions a CTA claims per atomic, 1..64 */
    int32_t pinned;          /* output only: 1 when efm_batch_set_tuning chose it */
    float sample_default_ms; /* output only: the tuning sample (up to 256 jobs, strided) in the untuned
                                configuration (8 warps, every CTA an SM holds, input order, tile 32,
                                chunk 1); 0 when no search ran */
    float sample_tuned_ms;   /* output only: the same sample in the chosen configuration */
} efm_batch_tune;

/* The configuration the last batch ran with.  A batch of at least 64 jobs
 * whose shape (log2 jobs, largest row class, SM count) has not been seen
 * times a sample of its jobs: CTAs per SM and queue order, then warps per
 * job, then the tile, then the queue chunk, each keeping the fastest.
 * EFM_EINVAL before any batch ran or for a null pointer. */
int efm_batch_tuning(efm_batch_tune *out);

/* Pin the configuration of later batches (the output-only fields are
 * ignored), or, with NULL, return to the search.  EFM_EINVAL for a value
 * outside the ranges above. */
int efm_batch_set_tuning(const efm_batch_tune *cfg);

/* Copy the results of target number `job_target_idx` (0-based position in
 * the targets array) into `supports` (host memory, capacity rows of W
 * words), sorted by (|U|, ascending column list).  supports == NULL is a
 * size query: *n_out receives the row count.  Rows beyond `capacity` are
 * not written (EFM_ECAPACITY is returned and *n_out holds the count).
 * words_per_set and ctr may be NULL.  Returns the target's warning flags. */
int efm_fetch_results(efm_job *job, int32_t job_target_idx, uint64_t *supports, int64_t capacity,
                      int64_t *n_out, int32_t *words_per_set, efm_counters *ctr);

/* Measurements of one target's traversal, for the benchmark's roofline:
 *  total_ms          device time of the whole traversal (CUDA events on the
 *                    network's stream, seeds to sorted results)
 *  expand_ms         summed device time of the expansion launches: the
 *                    generate kernel and the passes that finish its level
 *                    (prune, row, settle and dedup passes), event to event
 *  expand_launches   number of expansion launches (one per level, or per
 *                    chunk of a first-K level)
 *  expand_bytes      algorithmic bytes those launches must move: each parent
 *                    state read once, each new distinct state written once
 *                    (state = 8 W + 4 M + 4 bytes), 16 bytes of hash slot
 *                    traffic per child
 *  kernel_launches   every kernel this library launched for the target
 * Any output pointer may be NULL. */
int efm_job_timing(const efm_job *job, int32_t job_target_idx, double *total_ms, double *expand_ms,
                   int64_t *expand_launches, double *expand_bytes, int64_t *kernel_launches);

void efm_free_job(efm_job *job);
void efm_free_net(efm_net *net);

/* Sort supports into the output order of efm_fetch_results (by |U|, then
 * ascending column list) WITHOUT allocating any memory.  The paper has no
 * counterpart; this is for callers that cannot allocate where they sort:
 * code whose device memory is owned by another framework's allocator (a
 * private cudaMalloc would escape its accounting), or loops that must never
 * wait on an allocator.
 *  supports_in   device pointer, n_rows x words_per_set uint64 (caller-owned)
 *  supports_out  device pointer, same size; its bytes must not overlap the
 *                input's
 *  cuda_stream   stream the sort runs on (asynchronous; no host sync)
 * The only scratch, an index array, is a file-scope device array of
 * EFM_NOALLOC_MAX_ROWS entries (4 MiB) held by every GPU that loads the
 * library until exit.  All calls share it: calls whose GPU work overlaps
 * (unordered streams) race and may return wrong orders.  The first call on
 * a device (and the first after its context changed) looks up the array's
 * address in the current context; make it before any stream capture.
 * Errors: EFM_ECAPACITY if n_rows > EFM_NOALLOC_MAX_ROWS; EFM_EINVAL for
 * words_per_set outside 1..64, NULL or overlapping buffers; EFM_ECUDA. */
#define EFM_NOALLOC_MAX_ROWS (1 << 20)
int efm_sort_supports_noalloc(const uint64_t *supports_in, int64_t n_rows, int32_t words_per_set,
                              uint64_t *supports_out, uintptr_t cuda_stream);

/* ---- learned proposal of first-K searches -------------------------------
 * A two-layer MLP scores the parents of each level of a first-K search
 * (efm_limits.first_k > 0, proposal = EFM_LEARNED); parents are expanded in
 * descending score.  The search's branch and bound is exact, so the model
 * changes the order and the time to the answer, never the answer.
 *   x (128 features, BF16) -> h = relu(W1 x) (256 units, FP32 accumulate on
 *   the tensor cores) -> s = w2 . h + b2 (FP32); the hidden layer's bias is
 *   the weight of feature 10, which is constant 1.
 * Features of a state: see the feature list in the library's kernel source
 * (counts of unbalanced metabolites, pivot degree, |U|, secondary steps,
 * lowest columns, the share of U flux-dependent for the pivot from the
 * DEPTHy tags of efm_dependent_reactions, a 64-bucket hashed embedding of
 * the support).
 * Training: binary cross-entropy of s against labels of traced states
 * (1 = the state's support lies inside a support of the search's answer),
 * positives weighted by pos_weight, Adam (0.9, 0.999, 1e-8).
 * Parameters are one FP32 array of EFM_MLP_PARAMS values:
 *   W1[256][128] (row = hidden unit), then w2[256], then b2.
 * Not thread-safe; every call runs on the model's stream and returns when
 * its work is done.  Errors: EFM_EINVAL (bad arguments), EFM_ENOMEM,
 * EFM_ECUDA, EFM_ETIMEOUT (a bounded device wait gave up). */
#define EFM_MLP_FEATURES 128
#define EFM_MLP_HIDDEN 256
#define EFM_MLP_PARAMS (256 * 128 + 256 + 1)

/* New model with seeded uniform fan-in initialisation (splitmix64 stream;
 * W1 in +-sqrt(6/128), w2 in +-sqrt(3/256), b2 = 0) and no training rows. */
int efm_model_create(uint64_t seed, uintptr_t cuda_stream, efm_model **out);

/* Read (write = 0) or replace (write = 1; resets the Adam state) the FP32
 * parameters; params is a host array of EFM_MLP_PARAMS floats.  Saving and
 * loading a model is reading and writing this array. */
int efm_model_params(efm_model *model, float *params, int32_t write);

/* Append n training rows: x host [n][128] FP32 (stored as BF16), y host [n]
 * labels, each 0 or 1. */
int efm_model_add_rows(efm_model *model, const float *x, const float *y, int64_t n);

/* Training rows held, and how many are labelled 1 (either may be NULL). */
int efm_model_rows(efm_model *model, int64_t *n_rows, int64_t *n_positive);
int efm_model_clear_rows(efm_model *model);

/* Scores of n host rows x [n][128] (rounded to BF16) into host scores[n],
 * through the tensor-core forward kernel. */
int efm_model_forward(efm_model *model, const float *x, int64_t n, float *scores);

/* Gradient of the mean training loss over all held rows (host grad of
 * EFM_MLP_PARAMS floats, same layout as the parameters) and the loss;
 * the parameters are not changed.  dL/dh is rounded to BF16 for the
 * tensor-core product dW1 = dH^T X. */
int efm_model_gradient(efm_model *model, float pos_weight, float *grad, float *loss);

/* Adam training over the held rows: `epochs` passes in seeded random order
 * of 128-row tiles, batch_tiles tiles per step.  last_loss: mean batch loss
 * of the last epoch (may be NULL). */
int efm_model_train(efm_model *model, int32_t epochs, int32_t batch_tiles, float lr, float pos_weight, uint64_t seed,
                    float *last_loss);

/* Training rows from traces: for each target, run the first-K search of
 * `limits` (first_k > 0, max_results = 0) in plain order, then run its last
 * deepening run again and record the features of up to rows_per_level states of every
 * level's frontier (an evenly strided sample), labelled 1 when the state's
 * support lies inside a support of the answer.  Targets whose search is
 * truncated or finds nothing add no rows. */
int efm_model_trace(efm_model *model, efm_net *net, const int32_t *targets, int32_t n_targets,
                    const efm_limits *limits, int64_t rows_per_level);

void efm_model_free(efm_model *model);

/* Human-readable name of a status code. */
const char *efm_status_str(int code);

/* Optional device allocator (e.g. PyTorch's caching allocator).  alloc
 * returns device memory of `bytes` usable on `stream` or NULL; free
 * releases it.  Passing NULL functions restores cudaMallocAsync /
 * cudaFreeAsync.  Set before loading networks. */
typedef void *(*efm_alloc_fn)(size_t bytes, uintptr_t stream, void *ctx);
typedef void (*efm_free_fn)(void *ptr, size_t bytes, uintptr_t stream, void *ctx);
int efm_set_allocator(efm_alloc_fn alloc, efm_free_fn free_fn, void *ctx);

#ifdef __cplusplus
}
#endif
#endif /* EFMGRAPH_H */
