// efm_internal.cuh -- shared declarations of the CUDA path (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/efmgraph.h"

namespace efm {

constexpr int kMaxW = 64;           // support words (EFM_MAX_COLUMNS / 64)
constexpr int kExpandWarps = 8;     // warps per CTA of the expansion kernel
constexpr int kAcceptWarps = 4;     // warps per CTA of the minimality kernel
constexpr unsigned long long kEmpty = ~0ull;
constexpr uint32_t kPending = 0xFFFFFFFFu;
constexpr uint32_t kOverflowIdx = 0xFFFFFFFEu;
constexpr int kNumPrimes = 24;
constexpr int kStageLimitBytes = 72 * 1024;  // static network staged in smem up to this size
constexpr int kStageSparseLimitBytes = 100 * 1024;  // generic kernel: its sparse tables staged up to this size
constexpr int64_t kFirstKChunkMin = 8192;     // first-K search: fewest parents per expansion launch
constexpr int64_t kFirstKChunks = 32;         // first-K search: launches per level, at most
constexpr int64_t kResultWindow = 256;        // first-K search: new results fetched with the counters
constexpr int kWaitSpinLimit = 1 << 20;       // polls of a bounded device-side wait (with ~0.25 us sleeps)

// device error bits (ctr[C_ERR])
enum : unsigned { ERR_TIMEOUT = 1u, ERR_CAND_CAP = 2u, ERR_RES_CAP = 4u, ERR_TABLE_FULL = 8u,
                  ERR_PRIMES = 16u, ERR_LEN = 32u, ERR_WATCHDOG = 64u, ERR_BOUNDS = 128u };

// device counter block (unsigned long long each)
enum {
    C_LEVELS = 0, C_SEEDS, C_EXP, C_OVF, C_BAL, C_CAND, C_RES, C_PRUNED, C_FRONTIER, C_FRONTIER_MAX, C_STATUS,
    C_NEXT = 12,  // states allocated in the arena being written
    C_DEGSUM,     // sum of pivot degrees of the states written (children bound of the next level)
    C_CAND_N,     // candidate list length (cumulative)
    C_RES_N,      // result list length (cumulative)
    C_ERR,        // ERR_* bits
    C_WRITTEN,    // generate/dedup split: child rows reserved so far in the level
    C_UNWRITTEN,  // children whose row did not fit the child arena
    C_UNV,        // distinct fingerprints among the children without a row
    C_OUT_N = 20, // batched traversal: rows written to the job's output
    C_DONE,       // batched traversal: job finished
    C_ACC_BEGIN,  // first candidate the next device-range minimality launch judges
    C_DEDUP_BEGIN,  // first reserved row the next dedup launch examines
    C_DIAG = 24,  // first bounds/watchdog record: code, value, limit, level
    C_ZERO = 28,  // subtractive steps discarded: no positive flux left on the reaction (Prop. 3)
    C_SLOW,       // narrow networks: children handed to the settle pass in this launch
    C_LIVE,       // surviving rows counted by the live-list pass
    C_CAPDEAD,    // first-K: children at the length cap that can never balance
    C_COUNT = 32
};

// Static network, packed into one 16-byte aligned word array (the "blob").
// Packed entry: (index << 20) | (coefficient & 0xFFFFF), index < 4096,
// coefficient a signed 20-bit value.
struct NetView {
    const uint32_t *blob;  // device
    int blob_words;        // multiple of 4
    int M, N, W, Mpad, EPL;
    int o_colptr, o_colent;    // S_int by column: rows with coefficients
    int o_consptr, o_consent;  // per internal row: consuming columns, |coef|
    int o_prodptr, o_prodent;  // per internal row: producing columns, |coef|
    int o_twin;                // per column: twin column or -1 (as int32)
    int o_keypos, o_keyneg;    // per internal row: (degree << 16) | row
    int o_hbits;               // per column: ceil(log2(|S_int[:,k]|^2))
    int o_dcols;               // dense S_int by column: N rows of Mpad int32 (16-byte aligned)
    // narrow networks (M <= 64): state summary tables (see efm_netprep.h)
    int narrow;
    int o_rank;                // per row: rank in the positive key order | rank in the negative << 8
    int o_keyr;                // per rank: positive key [64], then negative key [64]
    int o_hrow;                // per row: 64-bit row hash constant R[m]
    int o_colx;                // per column: suppP, suppN, suppR, HC (u64 each), smax, gcd1 (10 words)
    // wide networks: per column, G lane masks of the rows it consumes, then
    // (at o_fixp) of the rows it produces, G = min(32, 4 EPL); 0: absent
    int o_fixc, o_fixp;
    const int32_t *metptr;     // full S rows over split columns (seeds), [n_met + 1]
    const uint32_t *metent;    // packed (column, coefficient)
    int n_met;
};

__host__ __device__ inline int ent_index(uint32_t e) { return (int)(e >> 20); }
__host__ __device__ inline int32_t ent_coef(uint32_t e) { return ((int32_t)(e << 12)) >> 12; }

// One arena of pathway states, structure of arrays.
struct Arena {
    uint64_t *U;     // [cap][W]
    int32_t *B;      // [cap][Mpad]
    uint32_t *meta;  // [cap]: pivot row | pivot degree << 10 | |U| << 23
    int64_t cap;
    // narrow networks: per-state summaries of the extra-flux row EF, kSumWords each
    //   sum[6 s + 0] = sum_m EF_m R[m] (mod 2^64), the linear row hash
    //   sum[6 s + 1] = positive entries, bit = rank of the row in the positive key order
    //   sum[6 s + 2] = negative entries, bit = rank of the row in the negative key order
    //   sum[6 s + 3] = rows with |EF_m| = 1
    //   sum[6 s + 4] = rows with odd EF_m
    //   sum[6 s + 5] = an upper bound of max_m |EF_m| (saturating at 2^31 - 1)
    uint64_t *sum;
    // first-K on wide networks: per state, 2G lane masks (G = min(32, 4 EPL)):
    // the rows some column of U consumes, then the rows some column of U
    // produces (null: not kept)
    uint32_t *fx;
};

constexpr int kSumWords = 6;

struct LevelArgs {
    Arena par;
    int64_t n_par;
    Arena child;
    unsigned long long *slots;  // state hash table
    uint64_t slot_mask;
    unsigned long long *cslots; // balanced-support hash table
    uint64_t cslot_mask;
    uint64_t *cand;             // [cand_cap][W]
    int64_t cand_cap;
    const uint64_t *res;        // [res_cap][W]
    const int32_t *bptr;        // [N + 1] result buckets by column
    const uint64_t *bres;       // bucket entries: the result's W support words (W <= 2)
    const int32_t *bids;        // bucket entries: result ids (W > 2), same buffer as bres
    const uint16_t *rcols;      // per result: column count, then its columns (stride kRcolStride)
    const uint64_t *band;       // W <= 2: per column, the intersection of the results containing it (or null)
    // W <= 2: the superset rule's index.  A result E is filed, for each of its
    // columns k, in cell (k, s) where s is E's other column with the fewest
    // results (its sentinel); a child adding k scans only the cells whose
    // sentinel lies in its support.  Null: the buckets above.
    const int32_t *cptr;        // [N * N + 1] cell offsets into cent
    const uint64_t *cent;       // cell entries: the result's W support words
    const uint64_t *cne;        // [N][W]: sentinels with a non-empty cell (k, s)
    const uint32_t *csingle;    // [N]: 1 if {k} itself is a result
    int level, max_len, max_sec;
    int cpw;                    // parents per warp chunk (1..32)
    unsigned long long *ctr;
    // first-K search (zero / null otherwise)
    const uint32_t *perm;       // parent order: position -> arena index (null: arena rows par_base + position)
    int64_t par_base;
    int fk_pc;                  // bound: |U| of the K-th smallest result found so far (0 = no bound)
    const uint64_t *fk_sup;     // bound: its support (W words)
    // first-K: drop an unbalanced child at the length cap that no sequence of
    // secondary steps can balance (0 = keep every child)
    int cap_dead;
    // generate/dedup split (single-job traversal): every surviving child gets
    // a reserved row and a fingerprint; the dedup pass keeps one per state
    uint64_t *fp;               // [fp_cap] fingerprint per reserved row (kDeadFp: unused)
    int64_t fp_cap;
    uint32_t *live;             // unused by the kernels (kept for the host's bookkeeping)
    int blk;                    // rows a warp reserves at a time (NG..32)
    // subtractive variant (Eq. 5): rows hold the extra flux (M entries), then
    // the flux of every column; a state's branches also take flux away from
    // a column in U, and its meta degree counts both lists of the pivot
    int sub;
    // narrow networks: children whose gcd or int32 range is not settled by
    // the summaries, kSlowWords words each, for the settle pass
    uint64_t *slow;
    int64_t slow_cap;
    // narrow networks: per reserved row, the row writer's record (parent row,
    // column | flags | |U| << 14, A, C); x = kNoRecord: nothing to write
    uint4 *wrec;
};

constexpr uint32_t kNoRecord = 0xFFFFFFFFu;

constexpr int kSlowWords = 8;

constexpr unsigned long long kDeadFp = ~0ull;  // fingerprint of a reserved row left unused

constexpr int kRcolStride = 65;  // column count + up to 64 columns per result
constexpr int kNarrowKeyRanks = 64;  // narrow networks: keys per rank order (efm_netprep.h kNarrowRows)
constexpr int kColxWordsDev = 10;    // narrow networks: per-column summary words (efm_netprep.h kColxWords)

struct AcceptArgs {
    const uint64_t *cand;
    int64_t cand_begin, cand_end;  // ignored when dev_range: [ctr[C_ACC_BEGIN], ctr[C_CAND_N]) instead
    int dev_range;
    int64_t cand_cap;
    uint64_t *res;
    uint16_t *rcols;            // written on accept when non-null
    int64_t res_cap;
    unsigned long long *ctr;
};

// Batched traversal: per-CTA scratch slice layout (byte offsets)
constexpr int kBatchThreads = 256;
struct BatchLayout {
    size_t slice_bytes;
    size_t o_U[2], o_B[2], o_meta[2];
    size_t o_slots, o_cslots, o_cand, o_res, o_bcnt, o_bfill, o_bptr, o_bres, o_sort, o_rcols;
    int64_t cap, cand_cap, res_cap;
    uint64_t slot_cap, cslot_cap;
};

struct BatchJob {
    NetView nv;
    int target, max_len;
    uint64_t *out;            // [res_cap][W] sorted supports
    unsigned long long *ctr;  // [C_COUNT] counters of this job (zeroed by the host)
};

struct BatchArgs {
    const BatchJob *jobs;
    const int *order;         // queue schedule: job index per queue position
    int n_jobs;
    unsigned int *queue;      // next queue position (zeroed by the host)
    char *pool;               // gridDim.x slices of layout.slice_bytes
    BatchLayout layout;
    int max_sec;
    int64_t max_frontier, max_results;
    int tile;                 // most parents a warp takes per pass (1..32)
    int chunk;                // queue positions a CTA claims at a time (>= 1)
};

// Learned proposal: MLP 128 -> 256 (ReLU) -> 1.  FP32 parameters in one
// buffer: W1 [256][128] (hidden unit, feature; the bias of the hidden layer
// is the weight of the constant feature), w2 [256], b2.
constexpr int kMlpFeatures = 128;
constexpr int kMlpHidden = 256;
constexpr int kMlpTileRows = 128;
constexpr int kMlpW1 = 0;
constexpr int kMlpW2 = kMlpHidden * kMlpFeatures;
constexpr int kMlpB2 = kMlpW2 + kMlpHidden;
constexpr int kMlpParams = kMlpB2 + 1;

// Byte offset of element (row, k) in a 128-column BF16 tile laid out as the
// K-major operand of tcgen05 without swizzling: 8 x 8 core matrices (8 rows
// of 16 bytes), 16 of them along K per group of 8 rows.
__host__ __device__ inline uint32_t mlp_blk_off(int row, int k)
{
    return (uint32_t)((((row >> 3) * 16 + (k >> 3)) * 128) + (row & 7) * 16 + (k & 7) * 2);
}

// kernels (efm_mlp.cu)
// map: frontier position -> arena row (null: identity); rows r take positions first + r * stride
cudaError_t launch_features(const NetView &nv, const Arena &par, const uint32_t *map, int64_t first, int64_t stride,
                            int64_t n, int level, int max_len, int max_sec, const uint64_t *dep, void *X, int64_t row0,
                            cudaStream_t s);
cudaError_t launch_labels(const uint64_t *U, int W, const uint32_t *map, int64_t first, int64_t stride, int64_t n,
                          const uint64_t *ans, int64_t n_ans, float *y, int64_t row0, cudaStream_t s);
cudaError_t launch_mlp_score(const void *X, int64_t n_rows, const void *wb, const float *params, float *score,
                             unsigned *err, cudaStream_t s);
cudaError_t launch_mlp_train(const void *X, const float *y, int64_t n_rows, const int32_t *tiles, int n_tiles,
                             const void *wb, const float *params, float pos_weight, float inv_n, float *grad,
                             float *loss, unsigned *err, cudaStream_t s);
cudaError_t launch_adam(float *params, float *grad, float *mom, float lr, int step, void *wb, cudaStream_t s);
cudaError_t launch_pack_w(const float *params, void *wb, cudaStream_t s);
// perm[i] = map[position of the i-th highest score] (map null: the position itself)
cudaError_t launch_score_order(const float *score, int64_t n, const uint32_t *map, unsigned *hist, uint32_t *perm,
                               cudaStream_t s);
cudaError_t launch_pack_rows(const float *x, int64_t n, void *X, int64_t row0, cudaStream_t s);
size_t mlp_score_smem();
size_t mlp_train_smem();

// kernels (efm_kernels.cu)
cudaError_t launch_seed(const NetView &nv, const LevelArgs &a, int target, cudaStream_t s);
// generate/dedup split of one expansion: children with rows and fingerprints,
// then one pass that keeps the first row of every distinct state
cudaError_t launch_generate(const NetView &nv, const LevelArgs &a, int grid, cudaStream_t s);
cudaError_t launch_dedup(const LevelArgs &a, int Mpad, int W, int sm_count, cudaStream_t s);
// narrow networks: settle the children the generate pass listed (exact gcd,
// int32 range, superset rule), then write their rows; a no-op otherwise
cudaError_t launch_settle(const NetView &nv, const LevelArgs &a, int sm_count, cudaStream_t s);
// narrow networks: the superset rule over the generate pass's reserved rows
cudaError_t launch_prune_rows(const NetView &nv, const LevelArgs &a, int sm_count, cudaStream_t s);
// narrow networks: write the extra-flux rows of the generate pass's children
cudaError_t launch_write_rows(const NetView &nv, const LevelArgs &a, int sm_count, cudaStream_t s);
// the surviving rows (meta != 0) of [0, n) appended to live; *count must be 0
cudaError_t launch_live_list(const uint32_t *meta, int64_t n, uint32_t *live, unsigned long long *count,
                             int sm_count, cudaStream_t s);
int generate_grid(const NetView &nv, int sm_count);
cudaError_t launch_accept(const NetView &nv, const AcceptArgs &a, cudaStream_t s);
// minimality test of the candidates appended since the last such launch (range read on the
// device, so no host round trip is needed between expansion and test); then advance the range
cudaError_t launch_accept_new(const NetView &nv, const AcceptArgs &a, int sm_count, cudaStream_t s);
cudaError_t launch_buckets(const NetView &nv, const uint64_t *res, int64_t n_res, int32_t *bcnt, int32_t *bptr,
                           int32_t *bfill, uint64_t *bres, uint64_t *band,
                           cudaStream_t s);  // W > 2: bres holds int32 ids; band (W <= 2, may be null)
// W <= 2: the sentinel index of the superset rule over results [0, n_res)
// (bcnt: results per column, from launch_buckets); ccnt/cfill: N*N scratch
cudaError_t launch_sentinel_index(const NetView &nv, const uint64_t *res, int64_t n_res, const int32_t *bcnt,
                                  int32_t *ccnt, int32_t *cfill, int32_t *cptr, uint64_t *cent, uint64_t *cne,
                                  uint32_t *csingle, cudaStream_t s);
cudaError_t launch_sort_results(const uint64_t *res, int64_t n, int W, uint32_t *idx, int64_t n_pow2,
                                uint64_t *out, int64_t n_keep, cudaStream_t s);
cudaError_t launch_iota(uint32_t *perm, int64_t n, cudaStream_t s);
cudaError_t launch_seedset(const NetView &nv, const LevelArgs &a, const int32_t *cols, int n_cols, cudaStream_t s);
cudaError_t launch_step_count(const NetView &nv, unsigned *r, cudaStream_t s);
cudaError_t launch_or_words(uint64_t *a, const uint64_t *b, int64_t n, cudaStream_t s);
cudaError_t launch_depthy(const NetView &nv, int L, unsigned r, unsigned long long n_paths, unsigned long long *dep_out,
                          unsigned long long *dep_in, int sm_count, cudaStream_t s);
// one thread waits on `flag` for kWaitSpinLimit polls; ERR_TIMEOUT in *err if it stays 0
cudaError_t launch_stalled_wait(const uint32_t *flag, unsigned long long *err, unsigned long long *polls,
                                cudaStream_t s);
cudaError_t launch_flux(const NetView &nv, const uint64_t *sup, int64_t n, int64_t *flux, int8_t *status, int sm_count,
                        cudaStream_t s);
cudaError_t launch_walks(const NetView &nv, const LevelArgs &a, int target, uint64_t seed, int64_t n_walks, int sm_count,
                         cudaStream_t s);
// the batched traversal runs `warps` warps per CTA (4 or 8), one job at a time
cudaError_t launch_batch(const BatchArgs &ba, int grid, int warps, cudaStream_t s);
int batch_blocks_per_sm(int warps);
size_t batch_smem_bytes(int warps);

}  // namespace efm
