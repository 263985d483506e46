// efm_api.cu -- the C-ABI: network preprocessing, the level loop driving the
// kernels, and result delivery.  Every step of the traversal runs in the
// kernels of efm_kernels.cu; this file only prepares static data, sizes
// buffers, launches and reads back one counter block per level.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstdio>
#include <map>
#include <mutex>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "efm_internal.cuh"
#include "efm_netprep.h"
#include "efm_topk.h"

static_assert(efm::kNarrowKeyRanks == efm::kNarrowRows && efm::kColxWordsDev == efm::kColxWords,
              "narrow-network table layout of the kernels and the loader");

using namespace efm;

namespace {

efm_alloc_fn g_alloc = nullptr;
efm_free_fn g_free = nullptr;
void *g_ctx = nullptr;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

bool dev_alloc(DevBuf &b, size_t bytes, cudaStream_t s)
{
    b.bytes = bytes ? bytes : 16;
    if (g_alloc) {
        b.p = g_alloc(b.bytes, (uintptr_t)s, g_ctx);
        return b.p != nullptr;
    }
    if (cudaMallocAsync(&b.p, b.bytes, s) != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return false;
    }
    return true;
}

void dev_free(DevBuf &b, cudaStream_t s)
{
    if (!b.p) return;
    if (g_free)
        g_free(b.p, b.bytes, (uintptr_t)s, g_ctx);
    else
        cudaFreeAsync(b.p, s);
    b.p = nullptr;
    b.bytes = 0;
}

uint64_t next_pow2(uint64_t x)
{
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

}  // namespace

struct efm_net {
    int n_met = 0, n_rxn = 0;
    cudaStream_t stream = nullptr;
    std::vector<int32_t> col_rxn;
    std::vector<int8_t> col_dir;
    NetView nv{};
    DevBuf blob, metptr, metent;
    // the subtractive traversal's view (rows of M + N entries: extra flux,
    // then flux per column), when M + N fits a row
    NetView nv_sub{};
    DevBuf blob_sub;
    bool has_sub = false;
    int sm_count = 0;
    DevBuf dep;             // DEPTHy tags (dep_out | dep_in) per internal metabolite, for the model's features
    bool dep_ready = false;
};

struct TargetOut {
    DevBuf sup;
    const uint64_t *borrowed = nullptr;  // batched jobs: rows inside the job's shared buffer
    int err = 0;                         // batched jobs: this job's error code (0 = none)
    int64_t n = 0;
    efm_counters ctr{};
    int status = 0;
    double total_ms = 0.0, expand_ms = 0.0, expand_bytes = 0.0;
    int64_t expand_launches = 0, kernel_launches = 0;
};

struct efm_job {
    efm_net *net = nullptr;
    std::vector<TargetOut> out;
    std::vector<int> words;  // batched jobs: support width of each entry
    DevBuf shared_out;       // batched jobs: output rows of every job
};

// Proposal model: FP32 parameters, their gradients and Adam moments, the
// BF16 operand copy of W1, and the training rows (BF16 feature tiles and
// labels) collected from traversal traces.
struct efm_model {
    cudaStream_t stream = nullptr;
    DevBuf params, grad, mom, wb, loss, err, X, y, tiles;
    int64_t n_rows = 0, cap_rows = 0;
    int step = 0;
};

extern "C" int efm_set_allocator(efm_alloc_fn alloc, efm_free_fn free_fn, void *ctx)
{
    if ((alloc == nullptr) != (free_fn == nullptr)) return EFM_EINVAL;
    g_alloc = alloc;
    g_free = free_fn;
    g_ctx = ctx;
    return EFM_OK;
}

extern "C" const char *efm_status_str(int code)
{
    switch (code) {
    case EFM_OK: return "ok";
    case EFM_EINVAL: return "invalid argument";
    case EFM_ENOMEM: return "out of memory";
    case EFM_ECAPACITY: return "device buffer capacity exceeded";
    case EFM_ETIMEOUT: return "bounded device wait expired";
    case EFM_ECUDA: return "CUDA runtime error";
    case EFM_EUNSUPPORTED: return "unsupported size";
    default: break;
    }
    if (code > 0) {
        switch (code & 7) {
        case EFM_TRUNCATED: return "completed: truncated";
        case EFM_CAPPED: return "completed: capped";
        case EFM_OVERFLOW_DROPPED: return "completed: overflow dropped";
        default: return "completed with warnings";
        }
    }
    return "unknown status";
}

extern "C" int efm_load_network(int32_t n_met, int32_t n_rxn, const int32_t *row_ptr, const int32_t *col_idx,
                                const int32_t *coef, const uint8_t *reversible, const uint8_t *external,
                                uintptr_t cuda_stream, efm_net **out)
{
    if (!out) return EFM_EINVAL;
    *out = nullptr;
    NetPrep prep;
    const int prc = prepare_network(n_met, n_rxn, row_ptr, col_idx, coef, reversible, external, prep);
    if (prc != EFM_OK) return prc;
    auto *net = new (std::nothrow) efm_net();
    if (!net) return EFM_ENOMEM;
    net->n_met = n_met;
    net->n_rxn = n_rxn;
    net->stream = (cudaStream_t)cuda_stream;
    net->col_rxn = prep.col_rxn;
    net->col_dir = prep.col_dir;
    const std::vector<uint32_t> &blob = prep.blob;
    const std::vector<int32_t> &mptr = prep.mptr;
    const std::vector<uint32_t> &ment = prep.ment;
    NetView &nv = net->nv;
    nv.o_colptr = prep.o_colptr;
    nv.o_colent = prep.o_colent;
    nv.o_consptr = prep.o_consptr;
    nv.o_consent = prep.o_consent;
    nv.o_prodptr = prep.o_prodptr;
    nv.o_prodent = prep.o_prodent;
    nv.o_twin = prep.o_twin;
    nv.o_keypos = prep.o_keypos;
    nv.o_keyneg = prep.o_keyneg;
    nv.o_hbits = prep.o_hbits;
    nv.o_dcols = prep.o_dcols;
    nv.narrow = prep.narrow ? 1 : 0;
    nv.o_rank = prep.o_rank;
    nv.o_keyr = prep.o_keyr;
    nv.o_hrow = prep.o_hrow;
    nv.o_colx = prep.o_colx;
    nv.o_fixc = prep.o_fixc;
    nv.o_fixp = prep.o_fixp;
    nv.blob_words = (int)blob.size();
    nv.M = prep.M;
    nv.N = prep.N;
    nv.W = prep.W;
    nv.EPL = prep.EPL;
    nv.Mpad = prep.Mpad;
    nv.n_met = n_met;
    cudaStream_t s = net->stream;
    int rc = EFM_OK;
    if (!dev_alloc(net->blob, blob.size() * 4, s) || !dev_alloc(net->metptr, mptr.size() * 4, s) ||
        !dev_alloc(net->metent, ment.size() * 4, s)) {
        rc = EFM_ENOMEM;
    } else if (cudaMemcpyAsync(net->blob.p, blob.data(), blob.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
               cudaMemcpyAsync(net->metptr.p, mptr.data(), mptr.size() * 4, cudaMemcpyHostToDevice, s) !=
                   cudaSuccess ||
               cudaMemcpyAsync(net->metent.p, ment.data(), ment.size() * 4, cudaMemcpyHostToDevice, s) !=
                   cudaSuccess ||
               cudaStreamSynchronize(s) != cudaSuccess) {
        rc = EFM_ECUDA;
    }
    int dev = 0;
    if (rc == EFM_OK && (cudaGetDevice(&dev) != cudaSuccess ||
                         cudaDeviceGetAttribute(&net->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess))
        rc = EFM_ECUDA;
    if (rc == EFM_OK && !g_alloc) {
        // keep freed arenas in this process's stream-ordered pool between jobs
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    }
    if (rc != EFM_OK) {
        cudaGetLastError();
        dev_free(net->blob, s);
        dev_free(net->metptr, s);
        dev_free(net->metent, s);
        delete net;
        return rc;
    }
    nv.blob = (const uint32_t *)net->blob.p;
    nv.metptr = (const int32_t *)net->metptr.p;
    nv.metent = (const uint32_t *)net->metent.p;
    // the subtractive view: the same static network with a dense copy whose
    // column k is S_int[:, k] followed by e_k
    NetPrep sub;
    if (prepare_network(n_met, n_rxn, row_ptr, col_idx, coef, reversible, external, sub, true) == EFM_OK) {
        if (!dev_alloc(net->blob_sub, sub.blob.size() * 4, s) ||
            cudaMemcpyAsync(net->blob_sub.p, sub.blob.data(), sub.blob.size() * 4, cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            dev_free(net->blob_sub, s);
            dev_free(net->blob, s);
            dev_free(net->metptr, s);
            dev_free(net->metent, s);
            delete net;
            return EFM_ENOMEM;
        }
        NetView &vs = net->nv_sub;
        vs = nv;
        vs.blob = (const uint32_t *)net->blob_sub.p;
        vs.blob_words = (int)sub.blob.size();
        vs.o_dcols = sub.o_dcols;
        vs.o_hbits = sub.o_hbits;
        vs.EPL = sub.EPL;
        vs.Mpad = sub.Mpad;
        vs.narrow = 0;
        vs.o_fixc = vs.o_fixp = 0;
        net->has_sub = true;
    }
    *out = net;
    return EFM_OK;
}

extern "C" int efm_network_shape(const efm_net *net, int32_t *n_columns, int32_t *words_per_set, int32_t *n_internal)
{
    if (!net) return EFM_EINVAL;
    if (n_columns) *n_columns = net->nv.N;
    if (words_per_set) *words_per_set = net->nv.W;
    if (n_internal) *n_internal = net->nv.M;
    return EFM_OK;
}

extern "C" int efm_column_map(const efm_net *net, int32_t *orig_rxn, int8_t *dir)
{
    if (!net) return EFM_EINVAL;
    for (int k = 0; k < net->nv.N; ++k) {
        if (orig_rxn) orig_rxn[k] = net->col_rxn[k];
        if (dir) dir[k] = net->col_dir[k];
    }
    return EFM_OK;
}

extern "C" void efm_free_net(efm_net *net)
{
    if (!net) return;
    cudaStream_t s = net->stream;
    dev_free(net->blob, s);
    dev_free(net->blob_sub, s);
    dev_free(net->metptr, s);
    dev_free(net->metent, s);
    dev_free(net->dep, s);
    cudaStreamSynchronize(s);
    delete net;
}

namespace {

// Device buffers of one traversal, reused across the targets of a job.
struct Work {
    DevBuf U[2], B[2], meta[2], live[2];
    DevBuf sum[2];  // narrow networks: per-state summaries of the extra-flux row
    DevBuf fx[2];   // first-K on wide networks: per-state lane masks of the rows U consumes / produces
    int fx_words = 0;  // lane-mask words per state (0: not kept)
    DevBuf slots, cslots, cand, res, bcnt, bfill, bptr, bres, ctr, sortidx, rcols;
    DevBuf fp;         // fingerprints of one level's reserved child rows
    DevBuf wrec;       // narrow networks: the row pass's record per reserved row (16 B)
    DevBuf slow;       // narrow networks: records of the children the settle pass decides
    int64_t slow_cap = 0;
    DevBuf perm, fkb;  // first-K search: parent order of a level, bound support
    DevBuf band;       // per column: intersection of the results containing it (W <= 2)
    DevBuf ccnt, cfill, cptr, cne, csingle, cent;  // W <= 2: the superset rule's sentinel index
    DevBuf lx, lscore, lhist, lerr;  // learned order: features, scores, buckets, error flag
    int64_t lx_rows = 0;
    int64_t rows[2] = {0, 0};  // capacity of each arena (rows)
    int64_t F_cap = 0, cand_cap = 0, res_cap = 0, bres_cap = 0;  // bres_cap in bucket entries
    int64_t fp_cap = 0, perm_cap = 0;
    uint64_t slot_cap = 0, cslot_cap = 0, sort_cap = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

void free_arena(Work &w, int i, cudaStream_t s)
{
    dev_free(w.U[i], s);
    dev_free(w.B[i], s);
    dev_free(w.meta[i], s);
    dev_free(w.live[i], s);
    dev_free(w.sum[i], s);
    dev_free(w.fx[i], s);
    w.rows[i] = 0;
}

void free_work(Work &w, cudaStream_t s)
{
    for (int i = 0; i < 2; ++i) free_arena(w, i, s);
    DevBuf *bufs[] = {&w.slots, &w.cslots, &w.cand, &w.res, &w.bcnt,    &w.bfill, &w.bptr,
                      &w.bres,  &w.ctr,    &w.sortidx, &w.rcols, &w.perm, &w.fkb,
                      &w.lx,    &w.lscore, &w.lhist,   &w.lerr, &w.band, &w.fp, &w.slow, &w.wrec,
                      &w.ccnt,  &w.cfill,  &w.cptr,    &w.cne,  &w.csingle, &w.cent};
    for (DevBuf *b : bufs) dev_free(*b, s);
    for (auto &e : w.ev)
        if (e) cudaEventDestroy(e);
}

// Arena i with room for `rows` states (contents are not kept).
bool alloc_arena(Work &w, const NetView &nv, int i, int64_t rows, cudaStream_t s)
{
    free_arena(w, i, s);
    const size_t F = (size_t)rows;
    bool ok = dev_alloc(w.U[i], F * nv.W * 8, s) && dev_alloc(w.B[i], F * nv.Mpad * 4, s) &&
              dev_alloc(w.meta[i], F * 4, s) && dev_alloc(w.live[i], F * 4, s);
    if (ok && nv.narrow) ok = dev_alloc(w.sum[i], F * kSumWords * 8, s);
    if (ok && w.fx_words) ok = dev_alloc(w.fx[i], F * w.fx_words * 4, s);
    if (ok) w.rows[i] = rows;
    return ok;
}

// The level's fingerprint array and state hash table hold `reserved` rows.
bool ensure_level_tables(Work &w, uint64_t reserved, cudaStream_t s)
{
    if ((int64_t)reserved > w.fp_cap) {
        dev_free(w.fp, s);
        dev_free(w.wrec, s);
        const int64_t cap = std::max<int64_t>((int64_t)reserved, w.fp_cap + w.fp_cap / 2);
        if (!dev_alloc(w.fp, (size_t)cap * 8, s) || !dev_alloc(w.wrec, (size_t)cap * 16, s)) return false;
        w.fp_cap = cap;
    }
    const uint64_t need = next_pow2(2 * reserved + 64);
    if (need > w.slot_cap) {
        dev_free(w.slots, s);
        if (!dev_alloc(w.slots, need * 8, s)) return false;
        w.slot_cap = need;
    }
    return true;
}

// The static network a traversal reads: the subtractive variant's rows
// carry the flux vector after the extra flux.
const NetView &view_of(const efm_net *net, const efm_limits &lim)
{
    return lim.variant == EFM_SUBTRACTIVE ? net->nv_sub : net->nv;
}

int alloc_work(Work &w, const efm_net *net, const efm_limits &lim, int total_warps, cudaStream_t s)
{
    const NetView &nv = view_of(net, lim);
    const int64_t default_cap = (int64_t)1 << 22;
    // a level writes a row for every surviving child before deduplication,
    // so an arena gets room for a budget-sized frontier plus duplicates and
    // the rows warps reserve but leave unused; a level that needs more is
    // run again with a larger arena
    w.F_cap = lim.max_frontier > 0 ? lim.max_frontier + 1 : default_cap;
    const int64_t rows = w.F_cap + w.F_cap / 8 + 32 * (int64_t)total_warps;
    w.cand_cap = (int64_t)1 << 20;
    w.res_cap = w.cand_cap;
    w.cslot_cap = next_pow2(2 * (uint64_t)w.cand_cap);
    // first-K on a wide network keeps the lane masks of the length-cap rule
    w.fx_words = (lim.first_k > 0 && nv.o_fixc > 0 && !nv.narrow) ? 2 * std::min(32, 4 * nv.EPL) : 0;
    const size_t W = (size_t)nv.W;
    bool ok = alloc_arena(w, nv, 0, rows, s) && alloc_arena(w, nv, 1, rows, s);
    ok = ok && ensure_level_tables(w, 1024 + 32 * (uint64_t)total_warps, s);
    ok = ok && dev_alloc(w.cslots, w.cslot_cap * 8, s);
    ok = ok && dev_alloc(w.cand, (size_t)w.cand_cap * W * 8, s);
    ok = ok && dev_alloc(w.res, (size_t)w.res_cap * W * 8, s);
    ok = ok && dev_alloc(w.bcnt, (size_t)nv.N * 4, s);
    ok = ok && dev_alloc(w.bfill, (size_t)nv.N * 4, s);
    ok = ok && dev_alloc(w.bptr, (size_t)(nv.N + 1) * 4, s);
    ok = ok && dev_alloc(w.ctr, C_COUNT * 8, s);
    if (nv.W > 2) ok = ok && dev_alloc(w.rcols, (size_t)w.res_cap * kRcolStride * 2, s);
    if (nv.W <= 2) {
        const size_t cells = (size_t)nv.N * nv.N;
        ok = ok && dev_alloc(w.band, (size_t)nv.N * nv.W * 8, s) && dev_alloc(w.ccnt, cells * 4, s) &&
             dev_alloc(w.cfill, cells * 4, s) && dev_alloc(w.cptr, (cells + 1) * 4, s) &&
             dev_alloc(w.cne, (size_t)nv.N * nv.W * 8, s) && dev_alloc(w.csingle, (size_t)nv.N * 4, s);
    }
    if (lim.first_k > 0) ok = ok && dev_alloc(w.fkb, W * 8, s);
    for (auto &e : w.ev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return EFM_ENOMEM;
    }
    return EFM_OK;
}

int err_from_bits(unsigned long long e)
{
    if (e & (ERR_TIMEOUT | ERR_WATCHDOG)) return EFM_ETIMEOUT;
    if (e & ERR_BOUNDS) return EFM_ECUDA;
    if (e & (ERR_CAND_CAP | ERR_RES_CAP | ERR_TABLE_FULL)) return EFM_ECAPACITY;
    if (e & (ERR_PRIMES | ERR_LEN)) return EFM_EUNSUPPORTED;
    return EFM_OK;
}

#define CK(x)                         \
    do {                              \
        if ((x) != cudaSuccess) {     \
            cudaGetLastError();       \
            return EFM_ECUDA;         \
        }                             \
    } while (0)

// The K smallest results found so far by a first-K search (output order:
// |U|, then the ascending column list), kept on the host; the K-th is the
// branch-and-bound of the next expansion launches.

// DEPTHy tags of the network for the model's features: the deepest walk
// length (at most 3) whose enumeration stays under 2^26 walks per
// metabolite; dep_out | dep_in per internal metabolite.  Computed once.
int ensure_dep_tags(efm_net *net)
{
    if (net->dep_ready) return EFM_OK;
    const NetView &nv = net->nv;
    cudaStream_t s = net->stream;
    const size_t words = (size_t)std::max(nv.M, 1) * nv.W;
    DevBuf r, din;
    unsigned rh = 0;
    int rc = EFM_OK;
    if (!dev_alloc(r, 4, s) || !dev_alloc(net->dep, words * 8, s) || !dev_alloc(din, words * 8, s)) rc = EFM_ENOMEM;
    if (rc == EFM_OK &&
        (cudaMemsetAsync(r.p, 0, 4, s) != cudaSuccess || launch_step_count(nv, (unsigned *)r.p, s) != cudaSuccess ||
         cudaMemcpyAsync(&rh, r.p, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess))
        rc = EFM_ECUDA;
    int depth = 0;
    unsigned long long n_paths = 1;
    while (rc == EFM_OK && rh > 0 && depth < 3 && n_paths * rh <= (1ull << 26)) {
        n_paths *= rh;
        ++depth;
    }
    if (rc == EFM_OK &&
        (cudaMemsetAsync(net->dep.p, 0, words * 8, s) != cudaSuccess || cudaMemsetAsync(din.p, 0, words * 8, s) != cudaSuccess ||
         (depth > 0 && launch_depthy(nv, depth, rh, n_paths, (unsigned long long *)net->dep.p,
                                     (unsigned long long *)din.p, net->sm_count, s) != cudaSuccess) ||
         launch_or_words((uint64_t *)net->dep.p, (const uint64_t *)din.p, (int64_t)words, s) != cudaSuccess))
        rc = EFM_ECUDA;
    dev_free(r, s);
    dev_free(din, s);
    if (rc != EFM_OK) {
        cudaGetLastError();
        dev_free(net->dep, s);
        return rc;
    }
    net->dep_ready = true;
    return EFM_OK;
}

// Training trace of a first-K search: features of a strided sample of each
// level's frontier, labelled against the search's answer.
struct Trace {
    efm_model *m = nullptr;
    const uint64_t *ans = nullptr;  // device, n_ans x W
    int64_t n_ans = 0;
    int64_t rows_per_level = 0;
};

bool model_reserve_rows(efm_model *m, int64_t rows);

// One (network, target) traversal.  Level 0 = seeds; level l expands F_{l-1}.
// With limits.first_k = K > 0 the traversal is the same, with each level's
// frontier expanded in chunks (in the order the proposal gives) and an exact
// branch and bound between chunks: once K results are known, a child that
// would follow the K-th of them in the output order is not generated, since
// every descendant keeps or grows its support.
// seedset (device, n_seedset columns): start from that one state instead of
// the target's seeds (Prop. 1), at level n_seedset - 1.
// A first-K sub-search that starts from rows [r0, r1) of another search's
// arena `par` (states of level `level`); deg_sum bounds their branch counts.
struct FrontierStart {
    Arena par;
    int64_t r0, r1;
    int level;
    uint64_t deg_sum;
};

// split_depth (first-K only): a level over the frontier budget does not end
// the search; its parents are split into parts, and the rest of the search
// runs from each part in turn, in a work area of its own (a part's levels may
// be split again while split_depth - 1 > 0).  A state reached from two parts
// is expanded twice, which changes no result: balanced supports are judged
// per part and merged, and the bound and the superset rule may use any
// accepted result.  fs / seed_top: such a part's start and the K smallest
// results known when it starts.
int run_target(efm_net *net, Work &w, const efm_limits &lim, int target, TargetOut &out,
               const efm_model *model = nullptr, Trace *trace = nullptr, const int32_t *seedset = nullptr,
               int n_seedset = 0, const FrontierStart *fs = nullptr, const std::vector<uint64_t> *seed_top = nullptr,
               int split_depth = 0)
{
    const NetView &nv = view_of(net, lim);
    cudaStream_t s = net->stream;
    const int grid = generate_grid(nv, net->sm_count);
    const int total_warps = grid * kExpandWarps;
    const int NG = 32 / std::min(32, std::max(4, 4 * nv.EPL));  // children per warp round
    unsigned long long *ctr = (unsigned long long *)w.ctr.p;
    unsigned long long h[C_COUNT];
    efm_counters &c = out.ctr;
    memset(&c, 0, sizeof(c));

    LevelArgs a{};
    a.cslots = (unsigned long long *)w.cslots.p;
    a.cslot_mask = w.cslot_cap - 1;
    a.cand = (uint64_t *)w.cand.p;
    a.cand_cap = w.cand_cap;
    a.res = (const uint64_t *)w.res.p;
    a.bptr = (const int32_t *)w.bptr.p;
    a.bres = nullptr;
    a.bids = nullptr;
    a.rcols = nv.W > 2 ? (const uint16_t *)w.rcols.p : nullptr;
    a.band = nv.W <= 2 ? (const uint64_t *)w.band.p : nullptr;
    a.max_len = lim.max_len;
    a.max_sec = lim.max_secondary;
    a.ctr = ctr;
    a.sub = lim.variant == EFM_SUBTRACTIVE ? 1 : 0;
    a.cap_dead = lim.first_k > 0 ? 1 : 0;
    auto arena = [&](int i) {
        Arena r{};
        r.U = (uint64_t *)w.U[i].p;
        r.B = (int32_t *)w.B[i].p;
        r.meta = (uint32_t *)w.meta[i].p;
        r.cap = w.rows[i];
        r.sum = (uint64_t *)w.sum[i].p;
        r.fx = (uint32_t *)w.fx[i].p;
        return r;
    };

    CK(cudaMemsetAsync(ctr, 0, C_COUNT * 8, s));
    CK(cudaMemsetAsync(w.cslots.p, 0xFF, w.cslot_cap * 8, s));
    CK(cudaMemsetAsync(w.bptr.p, 0, (size_t)(nv.N + 1) * 4, s));
    CK(cudaEventRecord(w.ev[0], s));

    // level 0: seeds (or the seed set's one state, at level |R_in| - 1),
    // written densely: the first level reads its parents in arena order
    int cur = 0;
    const int level0 = fs ? fs->level : (seedset ? n_seedset - 1 : 0);
    a.level = level0;
    a.child = arena(cur);
    if (fs) {
        // the first parents are the caller's rows: nothing to seed
    } else if (seedset) {
        CK(launch_seedset(nv, a, seedset, n_seedset, s));
    } else {
        CK(launch_seed(nv, a, target, s));
    }
    out.kernel_launches += fs ? 0 : 1;
    AcceptArgs acc{};
    acc.cand = (const uint64_t *)w.cand.p;
    acc.res = (uint64_t *)w.res.p;
    acc.res_cap = w.res_cap;
    acc.rcols = nv.W > 2 ? (uint16_t *)w.rcols.p : nullptr;
    acc.ctr = ctr;
    acc.cand_cap = w.cand_cap;
    auto read_ctr = [&]() -> int {
        if (cudaMemcpyAsync(h, ctr, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return EFM_ECUDA;
        }
        const int e = err_from_bits(h[C_ERR]);
        if (e != EFM_OK && getenv("EFM_DEBUG"))
            fprintf(stderr, "efm: device error bits %llx diag code %llu value %lld limit %lld level %lld\n",
                    h[C_ERR], h[C_DIAG], (long long)h[C_DIAG + 1], (long long)h[C_DIAG + 2],
                    (long long)h[C_DIAG + 3]);
        return e;
    };
    const bool fk = lim.first_k > 0;
    std::vector<uint64_t> window(fk ? (size_t)kResultWindow * nv.W : 0);
    TopK top;
    top.K = lim.first_k;
    top.W = nv.W;
    CK(launch_accept_new(nv, acc, net->sm_count, s));
    out.kernel_launches += 2;
    int rc = read_ctr();
    if (rc) return rc;
    int64_t res_n = (int64_t)std::min<unsigned long long>(h[C_RES_N], (unsigned long long)w.res_cap);
    if (fk && res_n > 0) {
        std::vector<uint64_t> fresh((size_t)res_n * nv.W);
        CK(cudaMemcpyAsync(fresh.data(), w.res.p, fresh.size() * 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        top.add(fresh.data(), res_n);
        if (top.pc > 0) CK(cudaMemcpyAsync(w.fkb.p, top.kth.data(), (size_t)nv.W * 8, cudaMemcpyHostToDevice, s));
    }
    if (fk && seed_top && !seed_top->empty()) {
        top.add(seed_top->data(), (int64_t)(seed_top->size() / nv.W));
        if (top.pc > 0) CK(cudaMemcpyAsync(w.fkb.p, top.kth.data(), (size_t)nv.W * 8, cudaMemcpyHostToDevice, s));
    }
    int64_t n_front = fs ? fs->r1 - fs->r0 : (int64_t)h[C_NEXT];  // distinct states of the level
    int64_t n_rows = n_front;              // arena rows the next level reads (seeds are dense)
    uint64_t deg_sum = fs ? fs->deg_sum : h[C_DEGSUM];
    int status = 0;
    bool split = false;  // the K smallest come from the parts of a split level (top)
    c.levels = 1;
    bool stop = false;
    if (lim.max_frontier > 0 && n_front > lim.max_frontier) {
        status |= EFM_TRUNCATED;
        stop = true;
    } else if (!fs && n_front > w.rows[cur]) {
        return EFM_ECAPACITY;
    } else {
        c.frontier += n_front;
        c.frontier_max = std::max<int64_t>(c.frontier_max, n_front);
        if (lim.max_results > 0 && (int64_t)h[C_RES] >= lim.max_results) {
            status |= EFM_CAPPED;
            stop = true;
        }
    }
    int64_t buckets_built_for = 0;
    float ms = 0.f;
    for (int level = level0 + 1; !stop && n_front > 0; ++level) {
        // every step adds a column or a secondary step, so depth is bounded
        if (level > lim.max_len + lim.max_secondary + 1) return EFM_ETIMEOUT;
        // buckets over every accepted result so far (all of them come from levels < `level`)
        if (res_n != buckets_built_for) {
            // bucket entries needed: sum of |E| <= res_n * max_len (grown on demand)
            const int64_t need = std::max<int64_t>(res_n * (int64_t)lim.max_len, 1);
            if (need > w.bres_cap) {
                dev_free(w.bres, s);
                dev_free(w.cent, s);
                const int64_t cap = std::max<int64_t>(need, 2 * w.bres_cap);
                if (!dev_alloc(w.bres, (size_t)cap * nv.W * 8, s)) return EFM_ENOMEM;
                if (nv.W <= 2 && !dev_alloc(w.cent, (size_t)cap * nv.W * 8, s)) return EFM_ENOMEM;
                w.bres_cap = cap;
            }
            a.bres = (const uint64_t *)w.bres.p;
            a.bids = (const int32_t *)w.bres.p;
            CK(launch_buckets(nv, (const uint64_t *)w.res.p, res_n, (int32_t *)w.bcnt.p, (int32_t *)w.bptr.p,
                              (int32_t *)w.bfill.p, (uint64_t *)w.bres.p, (uint64_t *)w.band.p, s));
            if (nv.W <= 2) {
                CK(launch_sentinel_index(nv, (const uint64_t *)w.res.p, res_n, (const int32_t *)w.bcnt.p,
                                         (int32_t *)w.ccnt.p, (int32_t *)w.cfill.p, (int32_t *)w.cptr.p,
                                         (uint64_t *)w.cent.p, (uint64_t *)w.cne.p, (uint32_t *)w.csingle.p, s));
                a.cptr = (const int32_t *)w.cptr.p;
                a.cent = (const uint64_t *)w.cent.p;
                a.cne = (const uint64_t *)w.cne.p;
                a.csingle = (const uint32_t *)w.csingle.p;
                out.kernel_launches += res_n > 0 ? 4 : 2;
            }
            out.kernel_launches += res_n > 0 ? 3 : 1;
            buckets_built_for = res_n;
        }
        if (trace && n_front > 0) {
            // training rows: a strided sample of this frontier (level - 1),
            // through the list of its surviving rows
            unsigned long long n_live = 0;
            CK(cudaMemsetAsync(ctr + C_LIVE, 0, 8, s));
            CK(launch_live_list((const uint32_t *)w.meta[cur].p, n_rows, (uint32_t *)w.live[cur].p, ctr + C_LIVE,
                                net->sm_count, s));
            CK(cudaMemcpyAsync(&n_live, ctr + C_LIVE, 8, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            const int64_t nl = (int64_t)n_live;
            const int64_t stride = std::max<int64_t>(1, (nl + trace->rows_per_level - 1) / trace->rows_per_level);
            const int64_t cnt = (nl + stride - 1) / stride;
            efm_model *m = trace->m;
            if (!model_reserve_rows(m, m->n_rows + cnt)) return EFM_ENOMEM;
            if ((rc = ensure_dep_tags(net))) return rc;
            const uint32_t *live = (const uint32_t *)w.live[cur].p;
            CK(launch_features(nv, arena(cur), live, 0, stride, cnt, level - 1, lim.max_len, lim.max_secondary,
                               (const uint64_t *)net->dep.p, m->X.p, m->n_rows, s));
            CK(launch_labels((const uint64_t *)w.U[cur].p, nv.W, live, 0, stride, cnt, trace->ans, trace->n_ans,
                             (float *)m->y.p, m->n_rows, s));
            m->n_rows += cnt;
        }
        // first-K: the level's parents in proposal order (positions -> arena
        // rows), expanded in chunks with the bound refreshed between them
        // (rows of later copies have no branches: they cost a meta read)
        const int64_t par_rows = n_rows;    // this level's parents
        const uint64_t par_deg = deg_sum;
        const bool ext = fs && level == level0 + 1;  // parents in the caller's arena
        int64_t chunk = n_rows;
        const uint32_t *order = nullptr;
        if (fk) {
            chunk = std::max<int64_t>(kFirstKChunkMin, (n_rows + kFirstKChunks - 1) / kFirstKChunks);
            if (model && lim.proposal == EFM_LEARNED && n_rows > chunk) {
                // the model's order: features of every parent, scores, and a
                // counting sort by score (highest first)
                const int64_t rows = (n_rows + kMlpTileRows - 1) / kMlpTileRows * kMlpTileRows;
                if (rows > w.lx_rows) {
                    dev_free(w.lx, s);
                    dev_free(w.lscore, s);
                    const int64_t cap = std::max<int64_t>(rows, 2 * w.lx_rows);
                    if (!dev_alloc(w.lx, (size_t)cap * kMlpFeatures * 2, s) || !dev_alloc(w.lscore, (size_t)cap * 4, s))
                        return EFM_ENOMEM;
                    w.lx_rows = cap;
                }
                if (n_rows > w.perm_cap) {
                    dev_free(w.perm, s);
                    const int64_t cap = std::max<int64_t>(n_rows, 2 * w.perm_cap);
                    if (!dev_alloc(w.perm, (size_t)cap * 4, s)) return EFM_ENOMEM;
                    w.perm_cap = cap;
                }
                if (!w.lhist.p) {
                    if (!dev_alloc(w.lhist, 4096 * 4, s) || !dev_alloc(w.lerr, 4, s)) return EFM_ENOMEM;
                    CK(cudaMemsetAsync(w.lerr.p, 0, 4, s));
                }
                if ((rc = ensure_dep_tags(net))) return rc;
                CK(launch_features(nv, arena(cur), nullptr, 0, 1, n_rows, level - 1, lim.max_len, lim.max_secondary,
                                   (const uint64_t *)net->dep.p, w.lx.p, 0, s));
                CK(launch_mlp_score(w.lx.p, n_rows, model->wb.p, (const float *)model->params.p,
                                    (float *)w.lscore.p, (unsigned *)w.lerr.p, s));
                CK(launch_score_order((const float *)w.lscore.p, n_rows, nullptr, (unsigned *)w.lhist.p,
                                      (uint32_t *)w.perm.p, s));
                order = (const uint32_t *)w.perm.p;
                out.kernel_launches += 6;
            }
        }
        // rows one warp reserves at a time: few for small or chunked levels
        // (a warp's unused reserved rows at the end of every launch are dead
        // weight in the arena), 32 for large ones
        const int64_t launches = (n_rows + chunk - 1) / chunk;
        const int blk = launches > 1 ? NG
                                     : (int)std::min<uint64_t>(32, std::max<uint64_t>((uint64_t)NG,
                                                                                     deg_sum / (64ull * total_warps)));
        const uint64_t reserved = deg_sum + (uint64_t)launches * blk * total_warps + 64;
        if (!ensure_level_tables(w, reserved, s)) return EFM_ENOMEM;
        // narrow networks: room for every child of a launch in the settle list
        const int64_t slow_need = (int64_t)deg_sum + 32 * (int64_t)total_warps + 64;  // + unused pool slots
        if (nv.narrow && slow_need > w.slow_cap) {
            dev_free(w.slow, s);
            const int64_t cap = std::max<int64_t>(slow_need, w.slow_cap + w.slow_cap / 2);
            if (!dev_alloc(w.slow, (size_t)cap * kSlowWords * 8, s)) return EFM_ENOMEM;
            w.slow_cap = cap;
        }
        const uint64_t nslots = next_pow2(2 * reserved + 64);
        unsigned long long snap[C_COUNT];
        memcpy(snap, h, sizeof(h));
        const int64_t n_front_level = n_front;  // distinct parents of this level
        // the level, run again with a larger child arena if some children
        // found no row and the fingerprints alone cannot show a truncation
        for (int attempt = 0;; ++attempt) {
            if (attempt > 4) return EFM_ECAPACITY;
            CK(cudaMemsetAsync(w.slots.p, 0xFF, nslots * 8, s));
            CK(cudaMemsetAsync(ctr + C_NEXT, 0, 2 * 8, s));
            CK(cudaMemsetAsync(ctr + C_WRITTEN, 0, 3 * 8, s));
            CK(cudaMemsetAsync(ctr + C_DEDUP_BEGIN, 0, 8, s));
            a.par = ext ? fs->par : arena(cur);
            a.child = arena(cur ^ 1);
            a.live = (uint32_t *)w.live[cur ^ 1].p;
            a.slots = (unsigned long long *)w.slots.p;
            a.slot_mask = nslots - 1;
            a.fp = (uint64_t *)w.fp.p;
            a.fp_cap = w.fp_cap;
            a.wrec = (uint4 *)w.wrec.p;
            a.blk = blk;
            a.slow = nv.narrow ? (uint64_t *)w.slow.p : nullptr;
            a.slow_cap = nv.narrow ? w.slow_cap : 0;
            a.level = level;
            unsigned long long exp_before = h[C_EXP];
            uint64_t next_before = 0;
            for (int64_t c0 = 0; c0 < n_rows; c0 += chunk) {
                const int64_t cn = std::min<int64_t>(chunk, n_rows - c0);
                a.n_par = cn;
                a.perm = order ? order + c0 : nullptr;
                a.par_base = order ? 0 : c0 + (ext ? fs->r0 : 0);
                a.cpw = (int)std::min<int64_t>(32, std::max<int64_t>(1, (cn + total_warps - 1) / total_warps));
                a.fk_pc = fk ? top.pc : 0;
                a.fk_sup = (const uint64_t *)w.fkb.p;
                a.max_len = (fk && top.pc > 0) ? std::min(lim.max_len, top.pc) : lim.max_len;
                CK(cudaEventRecord(w.ev[2], s));
                CK(cudaMemsetAsync(ctr + C_SLOW, 0, 8, s));
                CK(launch_generate(nv, a, grid, s));
                CK(launch_prune_rows(nv, a, net->sm_count, s));
                CK(launch_write_rows(nv, a, net->sm_count, s));
                CK(launch_settle(nv, a, net->sm_count, s));
                CK(launch_dedup(a, nv.Mpad, nv.W, net->sm_count, s));
                CK(cudaEventRecord(w.ev[3], s));
                // minimality test of the new candidates, range taken on the device
                CK(launch_accept_new(nv, acc, net->sm_count, s));
                // one round trip per chunk: the counters and, in a first-K search, a
                // window of the results that follow the ones already seen
                const int64_t win = fk ? std::min<int64_t>(kResultWindow, w.res_cap - res_n) : 0;
                if (win > 0)
                    CK(cudaMemcpyAsync(window.data(), (const uint64_t *)w.res.p + (size_t)res_n * nv.W,
                                       (size_t)win * nv.W * 8, cudaMemcpyDeviceToHost, s));
                if ((rc = read_ctr())) return rc;
                CK(cudaEventElapsedTime(&ms, w.ev[2], w.ev[3]));
                out.expand_ms += ms;
                out.expand_launches += 1;
                out.kernel_launches += nv.narrow ? (nv.W <= 2 && a.cptr ? 8 : 7) : 5;
                {
                    const double state_bytes = 8.0 * nv.W + 4.0 * nv.M + 4.0;
                    const uint64_t next_now = h[C_NEXT];
                    const double n_new = (double)(next_now - next_before);
                    const double n_child = (double)(h[C_EXP] - exp_before);
                    // distinct parents of the chunk (its rows include later copies
                    // and unused rows, which carry no state)
                    const double n_par = (double)cn * (double)n_front_level / (double)std::max<int64_t>(n_rows, 1);
                    out.expand_bytes += state_bytes * (n_par + n_new) + 16.0 * n_child;
                    if (getenv("EFM_DEBUG"))
                        fprintf(stderr,
                                "efm: level %d parents %lld items %llu children %.0f new %.0f rows %llu settled %llu "
                                "pruned %llu bytes %.0f ms %.3f\n",
                                level, (long long)cn, (unsigned long long)(c0 == 0 && chunk >= n_rows ? deg_sum : 0),
                                n_child, n_new, h[C_WRITTEN], h[C_SLOW], h[C_PRUNED],
                                state_bytes * (n_par + n_new) + 16.0 * n_child, ms);
                    exp_before = h[C_EXP];
                    next_before = next_now;
                }
                const int64_t res_now = (int64_t)std::min<unsigned long long>(h[C_RES_N], (unsigned long long)w.res_cap);
                if (fk && res_now > res_n) {
                    // the new results (beyond the window: fetched now) tighten the bound
                    const uint64_t *fresh = window.data();
                    std::vector<uint64_t> more;
                    if (res_now - res_n > win) {
                        more.resize((size_t)(res_now - res_n) * nv.W);
                        CK(cudaMemcpyAsync(more.data(), (const uint64_t *)w.res.p + (size_t)res_n * nv.W,
                                           more.size() * 8, cudaMemcpyDeviceToHost, s));
                        CK(cudaStreamSynchronize(s));
                        fresh = more.data();
                    }
                    const int pc_before = top.pc;
                    const std::vector<uint64_t> kth_before = top.kth;
                    top.add(fresh, res_now - res_n);
                    if (top.pc > 0 && (top.pc != pc_before || top.kth != kth_before))
                        CK(cudaMemcpyAsync(w.fkb.p, top.kth.data(), (size_t)nv.W * 8, cudaMemcpyHostToDevice, s));
                }
                res_n = res_now;
            }
            if (h[C_UNWRITTEN] == 0) break;  // every child has its row: the level is exact
            // some children found no row: their distinct fingerprints and the
            // distinct written rows bound |F_l| from below
            if (lim.max_frontier > 0 && (int64_t)(h[C_NEXT] + h[C_UNV]) > lim.max_frontier) break;
            // not decided: grow the child arena to every reserved row and run
            // the level again (its balanced supports are already judged, so
            // only the per-child counters are rolled back)
            if (!alloc_arena(w, nv, cur ^ 1, (int64_t)h[C_WRITTEN] + (int64_t)h[C_WRITTEN] / 8 + 1024, s))
                return EFM_ENOMEM;
            const int back[] = {C_EXP, C_OVF, C_BAL, C_PRUNED};
            for (int i : back) {
                h[i] = snap[i];
                CK(cudaMemcpyAsync(ctr + i, &snap[i], 8, cudaMemcpyHostToDevice, s));
            }
            CK(cudaStreamSynchronize(s));
        }
        const bool unwritten = h[C_UNWRITTEN] != 0;
        n_front = unwritten ? (int64_t)(h[C_NEXT] + h[C_UNV]) : (int64_t)h[C_NEXT];
        n_rows = (int64_t)std::min<unsigned long long>(h[C_WRITTEN], (unsigned long long)w.rows[cur ^ 1]);
        deg_sum = h[C_DEGSUM];
        c.levels = level - level0 + 1;
        cur ^= 1;
        if (lim.max_frontier > 0 && n_front > lim.max_frontier) {
            if (!(fk && split_depth > 0 && par_rows > 1)) {
                status |= EFM_TRUNCATED;
                break;
            }
            // first-K: the level's parents in parts of about half the
            // budget's worth of children, each run to the end
            Work w2;
            int rc2 = alloc_work(w2, net, lim, total_warps, s);
            if (rc2 == EFM_ENOMEM) {
                // no room for a second work area: the answer stays uncertified
                free_work(w2, s);
                cudaGetLastError();
                status |= EFM_TRUNCATED;
                break;
            }
            const int64_t parts = std::min<int64_t>(
                par_rows, std::max<int64_t>(2, (2 * n_front + lim.max_frontier - 1) / lim.max_frontier));
            // the level's parents: this search's arena, or the caller's rows
            // when the level is a part's first
            const Arena par_arena = ext ? fs->par : arena(cur ^ 1);
            const int64_t par0 = ext ? fs->r0 : 0;
            for (int64_t p = 0; rc2 == EFM_OK && p < parts; ++p) {
                FrontierStart sub{par_arena, par0 + par_rows * p / parts, par0 + par_rows * (p + 1) / parts, level - 1,
                                  par_deg};
                if (sub.r1 <= sub.r0) continue;
                TargetOut so;
                const std::vector<uint64_t> known = top.rows;
                rc2 = run_target(net, w2, lim, target, so, nullptr, nullptr, nullptr, 0, &sub, &known, split_depth - 1);
                if (rc2 == EFM_OK) {
                    status |= so.status;
                    if (so.n > 0) {
                        std::vector<uint64_t> got((size_t)so.n * nv.W);
                        if (cudaMemcpyAsync(got.data(), so.sup.p, got.size() * 8, cudaMemcpyDeviceToHost, s) !=
                                cudaSuccess ||
                            cudaStreamSynchronize(s) != cudaSuccess)
                            rc2 = EFM_ECUDA;
                        else
                            top.add(got.data(), so.n);
                    }
                    c.expansions += so.ctr.expansions;
                    c.overflow += so.ctr.overflow;
                    c.balanced += so.ctr.balanced;
                    c.pruned += so.ctr.pruned;
                    c.candidates += so.ctr.candidates;
                    c.results += so.ctr.results;
                    c.frontier_max = std::max<int64_t>(c.frontier_max, so.ctr.frontier_max);
                    c.levels = std::max<int64_t>(c.levels, so.ctr.levels + (level - 1 - level0));
                    out.expand_ms += so.expand_ms;
                    out.expand_bytes += so.expand_bytes;
                    out.expand_launches += so.expand_launches;
                    out.kernel_launches += so.kernel_launches;
                    if (getenv("EFM_DEBUG"))
                        fprintf(stderr, "efm: split level %d part %lld/%lld rows %lld status %d kept %lld\n", level,
                                (long long)p, (long long)parts, (long long)(sub.r1 - sub.r0), so.status,
                                (long long)(top.rows.size() / nv.W));
                }
                dev_free(so.sup, s);
                if (status & EFM_TRUNCATED) break;  // a part over the budget: the answer is uncertified anyway
            }
            free_work(w2, s);
            if (rc2) return rc2;
            split = true;
            break;
        }
        if (unwritten) return EFM_ECAPACITY;  // unreachable: the loop above runs such a level again
        c.frontier += n_front;
        c.frontier_max = std::max<int64_t>(c.frontier_max, n_front);
        if (lim.max_results > 0 && (int64_t)h[C_RES] >= lim.max_results) {
            status |= EFM_CAPPED;
            break;
        }
    }
    if ((int64_t)h[C_RES_N] > w.res_cap) return EFM_ECAPACITY;
    if (w.lerr.p) {
        unsigned e = 0;
        CK(cudaMemcpyAsync(&e, w.lerr.p, 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (e) return EFM_ETIMEOUT;
    }
    // output: sorted by (|U|, column list), capped
    int64_t n_keep = lim.max_results > 0 ? std::min<int64_t>(res_n, lim.max_results) : res_n;
    if (fk) n_keep = std::min<int64_t>(res_n, lim.first_k);
    if (split) {
        // the K smallest distinct supports of this search and its parts, sorted by TopK
        n_keep = (int64_t)(top.rows.size() / nv.W);
        if (!dev_alloc(out.sup, (size_t)std::max<int64_t>(n_keep, 1) * nv.W * 8, s)) return EFM_ENOMEM;
        if (n_keep > 0) CK(cudaMemcpyAsync(out.sup.p, top.rows.data(), top.rows.size() * 8, cudaMemcpyHostToDevice, s));
    } else {
        const uint64_t n2 = next_pow2((uint64_t)std::max<int64_t>(res_n, 1));
        if (n2 > w.sort_cap) {
            dev_free(w.sortidx, s);
            if (!dev_alloc(w.sortidx, n2 * 4, s)) return EFM_ENOMEM;
            w.sort_cap = n2;
        }
        if (!dev_alloc(out.sup, (size_t)std::max<int64_t>(n_keep, 1) * nv.W * 8, s)) return EFM_ENOMEM;
        CK(launch_sort_results((const uint64_t *)w.res.p, res_n, nv.W, (uint32_t *)w.sortidx.p, (int64_t)n2,
                               (uint64_t *)out.sup.p, n_keep, s));
        if (res_n > 0 && n_keep > 0) {
            int lg = 0;
            while ((1ull << lg) < n2) ++lg;
            out.kernel_launches += 2 + (int64_t)lg * (lg + 1) / 2;
        }
    }
    CK(cudaEventRecord(w.ev[1], s));
    CK(cudaEventSynchronize(w.ev[1]));
    CK(cudaEventElapsedTime(&ms, w.ev[0], w.ev[1]));
    out.total_ms = ms;
    out.n = n_keep;
    // (the parts of a split level have added their own work already)
    c.seeds = (int64_t)h[C_SEEDS];
    c.expansions += (int64_t)h[C_EXP];
    c.overflow += (int64_t)h[C_OVF];
    c.balanced += (int64_t)h[C_BAL];
    c.candidates += (int64_t)h[C_CAND_N];
    c.results += (int64_t)h[C_RES];
    c.pruned += (int64_t)h[C_PRUNED];
    c.zero_flux = (int64_t)h[C_ZERO];
    if (c.overflow) status |= EFM_OVERFLOW_DROPPED;
    c.status = status;
    out.status = status;
    return EFM_OK;
}

// levels of a first-K search that may be split inside one another.  Two
// certified 156 of the 192 held-out genome targets at K = 1000 against 141
// for one, in 2.7 times the time (most of it on the few hardest targets).
constexpr int kFirstKSplitDepth = 1;

// First-K by deepening the length cap.  The results of size <= P are exactly
// the results of the traversal run with max_len = P (every state on a path to
// such a result is no larger), so runs at P = 1, 2, ... stop at the first P
// with at least K results, or at limits.max_len.  The cap keeps each run's
// levels to states of size <= P and lets the length-cap rule drop the states
// that can no longer balance.  A run that overflows the frontier budget ends
// the search uncertified (TRUNCATED).  The counters are the last run's; the
// timings add up every run.  *depth: the P of the last run.  A seed set
// (Prop. 1) starts the deepening at its own size.
int run_first_k(efm_net *net, Work &w, const efm_limits &lim, int target, TargetOut &out, const efm_model *model,
                int *depth, const int32_t *seedset = nullptr, int n_seedset = 0)
{
    double total_ms = 0.0, expand_ms = 0.0, expand_bytes = 0.0;
    int64_t expand_launches = 0, kernel_launches = 0;
    for (int P = std::max(1, n_seedset);; ++P) {
        efm_limits l2 = lim;
        l2.max_len = std::min(P, lim.max_len);
        TargetOut o;
        const int rc = run_target(net, w, l2, target, o, model, nullptr, seedset, n_seedset, nullptr, nullptr,
                                  kFirstKSplitDepth);
        if (rc) {
            dev_free(o.sup, net->stream);
            return rc;
        }
        total_ms += o.total_ms;
        expand_ms += o.expand_ms;
        expand_bytes += o.expand_bytes;
        expand_launches += o.expand_launches;
        kernel_launches += o.kernel_launches;
        if ((o.status & EFM_TRUNCATED) || o.n >= lim.first_k || P >= lim.max_len) {
            out = o;
            out.total_ms = total_ms;
            out.expand_ms = expand_ms;
            out.expand_bytes = expand_bytes;
            out.expand_launches = expand_launches;
            out.kernel_launches = kernel_launches;
            if (depth) *depth = l2.max_len;
            return EFM_OK;
        }
        dev_free(o.sup, net->stream);
    }
}

}  // namespace

extern "C" int efm_find_pathways(efm_net *net, const int32_t *targets, int32_t n_targets, const efm_limits *limits,
                                 const efm_model *model, efm_job **out)
{
    if (!out) return EFM_EINVAL;
    *out = nullptr;
    if (!net || !targets || n_targets <= 0 || !limits) return EFM_EINVAL;
    const efm_limits lim = *limits;
    if (lim.max_len < 1 || lim.max_len > EFM_MAX_LEN || lim.max_secondary < 0 || lim.first_k < 0 ||
        (lim.proposal != EFM_PLAIN && lim.proposal != EFM_LEARNED))
        return EFM_EINVAL;
    if (lim.first_k > 0 && lim.max_results != 0) return EFM_EINVAL;
    if (lim.max_frontier > ((int64_t)1 << 31)) return EFM_EINVAL;  // arena indices are 32-bit
    if ((lim.variant != EFM_ADDITIVE && lim.variant != EFM_SUBTRACTIVE) || lim.reserved != 0) return EFM_EINVAL;
    if (lim.variant == EFM_SUBTRACTIVE && (lim.first_k != 0 || lim.proposal != EFM_PLAIN)) return EFM_EINVAL;
    if (lim.variant == EFM_SUBTRACTIVE && !net->has_sub) return EFM_EUNSUPPORTED;
    // a model orders a first-K search and nothing else
    if ((lim.proposal == EFM_LEARNED) != (model != nullptr) || (model && lim.first_k <= 0)) return EFM_EINVAL;
    const efm_model *mdl = model;
    for (int i = 0; i < n_targets; ++i)
        if (targets[i] < -1 || targets[i] >= net->n_met) return EFM_EINVAL;
    auto *job = new (std::nothrow) efm_job();
    if (!job) return EFM_ENOMEM;
    job->net = net;
    job->out.resize(n_targets);
    Work w;
    const int total_warps = generate_grid(view_of(net, lim), net->sm_count) * kExpandWarps;
    int rc = alloc_work(w, net, lim, total_warps, net->stream);
    int flags = 0;
    for (int i = 0; rc == EFM_OK && i < n_targets; ++i) {
        rc = lim.first_k > 0 ? run_first_k(net, w, lim, targets[i], job->out[i], mdl, nullptr)
                             : run_target(net, w, lim, targets[i], job->out[i], mdl);
        flags |= job->out[i].status;
    }
    free_work(w, net->stream);
    if (cudaStreamSynchronize(net->stream) != cudaSuccess && rc == EFM_OK) rc = EFM_ECUDA;
    if (rc != EFM_OK) {
        cudaGetLastError();
        efm_free_job(job);
        return rc;
    }
    *out = job;
    return flags;
}

extern "C" int efm_find_pathways_from(efm_net *net, const int32_t *columns, int32_t n_columns,
                                      const efm_limits *limits, efm_job **out)
{
    if (!out) return EFM_EINVAL;
    *out = nullptr;
    if (!net || !columns || !limits) return EFM_EINVAL;
    const efm_limits lim = *limits;
    if (lim.max_len < 1 || lim.max_len > EFM_MAX_LEN || lim.max_secondary < 0 || lim.first_k < 0 ||
        lim.proposal != EFM_PLAIN || (lim.first_k > 0 && lim.max_results != 0))
        return EFM_EINVAL;
    if ((lim.variant != EFM_ADDITIVE && lim.variant != EFM_SUBTRACTIVE) || lim.reserved != 0) return EFM_EINVAL;
    if (lim.variant == EFM_SUBTRACTIVE && lim.first_k != 0) return EFM_EINVAL;
    if (lim.variant == EFM_SUBTRACTIVE && !net->has_sub) return EFM_EUNSUPPORTED;
    if (n_columns < 1 || n_columns > lim.max_len) return EFM_EINVAL;
    for (int i = 0; i < n_columns; ++i) {
        if (columns[i] < 0 || columns[i] >= net->nv.N) return EFM_EINVAL;
        for (int j = 0; j < i; ++j) {
            const int a = columns[i], b = columns[j];
            const bool twins = net->col_rxn[a] == net->col_rxn[b];  // same reaction: the two directions
            if (a == b || twins) return EFM_EINVAL;
        }
    }
    auto *job = new (std::nothrow) efm_job();
    if (!job) return EFM_ENOMEM;
    job->net = net;
    job->out.resize(1);
    cudaStream_t s = net->stream;
    Work w;
    DevBuf cols;
    const int total_warps = generate_grid(view_of(net, lim), net->sm_count) * kExpandWarps;
    int rc = alloc_work(w, net, lim, total_warps, s);
    if (rc == EFM_OK && !dev_alloc(cols, (size_t)n_columns * 4, s)) rc = EFM_ENOMEM;
    if (rc == EFM_OK && cudaMemcpyAsync(cols.p, columns, (size_t)n_columns * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
        rc = EFM_ECUDA;
    if (rc == EFM_OK && lim.first_k > 0)
        rc = run_first_k(net, w, lim, -1, job->out[0], nullptr, nullptr, (const int32_t *)cols.p, n_columns);
    else if (rc == EFM_OK)
        rc = run_target(net, w, lim, -1, job->out[0], nullptr, nullptr, (const int32_t *)cols.p, n_columns);
    free_work(w, s);
    dev_free(cols, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == EFM_OK) rc = EFM_ECUDA;
    if (rc != EFM_OK) {
        cudaGetLastError();
        efm_free_job(job);
        return rc;
    }
    *out = job;
    return job->out[0].status;
}

extern "C" int efm_dependent_reactions(efm_net *net, int32_t depth, uint64_t *dep_out, uint64_t *dep_in,
                                       int32_t *steps_max, double *kernel_ms)
{
    if (!net || depth < 1 || depth > 16 || !dep_out || !dep_in) return EFM_EINVAL;
    cudaStream_t s = net->stream;
    const NetView &nv = net->nv;
    const size_t words = (size_t)std::max(nv.M, 1) * nv.W;
    DevBuf r, dout, din;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = EFM_OK;
    unsigned rh = 0;
    if (!dev_alloc(r, 4, s) || !dev_alloc(dout, words * 8, s) || !dev_alloc(din, words * 8, s)) rc = EFM_ENOMEM;
    if (rc == EFM_OK &&
        (cudaMemsetAsync(r.p, 0, 4, s) != cudaSuccess || launch_step_count(nv, (unsigned *)r.p, s) != cudaSuccess ||
         cudaMemcpyAsync(&rh, r.p, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess))
        rc = EFM_ECUDA;
    // r^depth walks per metabolite (Alg. 2 enumerates them all)
    unsigned long long n_paths = 1;
    for (int l = 0; rc == EFM_OK && l < depth; ++l) {
        if (rh == 0) {
            n_paths = 0;
            break;
        }
        if (n_paths > (1ull << 40) / rh) rc = EFM_EUNSUPPORTED;
        n_paths *= rh;
    }
    float ms = 0.f;
    if (rc == EFM_OK &&
        (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
         cudaMemsetAsync(dout.p, 0, words * 8, s) != cudaSuccess || cudaMemsetAsync(din.p, 0, words * 8, s) != cudaSuccess ||
         cudaEventRecord(e0, s) != cudaSuccess ||
         launch_depthy(nv, depth, rh, n_paths, (unsigned long long *)dout.p, (unsigned long long *)din.p, net->sm_count,
                       s) != cudaSuccess ||
         cudaEventRecord(e1, s) != cudaSuccess ||
         cudaMemcpyAsync(dep_out, dout.p, (size_t)nv.M * nv.W * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
         cudaMemcpyAsync(dep_in, din.p, (size_t)nv.M * nv.W * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
         cudaStreamSynchronize(s) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = EFM_ECUDA;
    if (rc == EFM_OK) {
        if (steps_max) *steps_max = (int32_t)rh;
        if (kernel_ms) *kernel_ms = ms;
    }
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(r, s);
    dev_free(dout, s);
    dev_free(din, s);
    return rc;
}

extern "C" int efm_flux_vectors(efm_net *net, const uint64_t *supports, int64_t n, int64_t *flux, int8_t *status)
{
    if (!net || n < 0 || (n > 0 && (!supports || !flux || !status))) return EFM_EINVAL;
    if (n == 0) return EFM_OK;
    cudaStream_t s = net->stream;
    const size_t W = (size_t)net->nv.W;
    DevBuf dsup, dflux, dst;
    int rc = EFM_OK;
    if (!dev_alloc(dsup, (size_t)n * W * 8, s) || !dev_alloc(dflux, (size_t)n * EFM_FLUX_COLUMNS * 8, s) ||
        !dev_alloc(dst, (size_t)n, s)) {
        rc = EFM_ENOMEM;
    } else if (cudaMemcpyAsync(dsup.p, supports, (size_t)n * W * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
               launch_flux(net->nv, (const uint64_t *)dsup.p, n, (int64_t *)dflux.p, (int8_t *)dst.p, net->sm_count,
                           s) != cudaSuccess ||
               cudaMemcpyAsync(flux, dflux.p, (size_t)n * EFM_FLUX_COLUMNS * 8, cudaMemcpyDeviceToHost, s) !=
                   cudaSuccess ||
               cudaMemcpyAsync(status, dst.p, (size_t)n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
               cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        rc = EFM_ECUDA;
    }
    dev_free(dsup, s);
    dev_free(dflux, s);
    dev_free(dst, s);
    return rc;
}

extern "C" int efm_check_bounded_wait(efm_net *net, int64_t *polls, double *waited_ms)
{
    if (!net) return EFM_EINVAL;
    cudaStream_t s = net->stream;
    DevBuf dbuf;  // flag (never set), padding, error word, poll count
    if (!dev_alloc(dbuf, 32, s)) return EFM_ENOMEM;
    unsigned long long h[2] = {0, 0};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = EFM_OK;
    auto *base = (unsigned long long *)dbuf.p;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaMemsetAsync(dbuf.p, 0, 32, s) != cudaSuccess || cudaEventRecord(e0, s) != cudaSuccess ||
        launch_stalled_wait((const uint32_t *)dbuf.p, base + 2, base + 3, s) != cudaSuccess ||
        cudaEventRecord(e1, s) != cudaSuccess ||
        cudaMemcpyAsync(h, base + 2, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        rc = EFM_ECUDA;
    } else {
        float ms = 0.f;
        if (waited_ms) *waited_ms = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess ? (double)ms : -1.0;
        if (polls) *polls = (int64_t)h[1];
        rc = err_from_bits(h[0]);  // the mapping every traversal's error word goes through
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(dbuf, s);
    return rc;
}

extern "C" int efm_sample_pathways(efm_net *net, int32_t target, const efm_limits *limits, uint64_t seed,
                                   int64_t n_walks, efm_job **out)
{
    if (!out) return EFM_EINVAL;
    *out = nullptr;
    if (!net || !limits || n_walks < 0) return EFM_EINVAL;
    efm_limits lim = *limits;
    if (lim.max_len < 1 || lim.max_len > EFM_MAX_LEN || lim.max_secondary < 0 || lim.max_secondary > 63 ||
        lim.first_k != 0 || lim.proposal != EFM_PLAIN || target < -1 || target >= net->n_met ||
        lim.variant != EFM_ADDITIVE || lim.reserved != 0)
        return EFM_EINVAL;
    lim.max_frontier = 1;  // walks keep their state in registers: no arenas
    cudaStream_t s = net->stream;
    const NetView &nv = net->nv;
    auto *job = new (std::nothrow) efm_job();
    if (!job) return EFM_ENOMEM;
    job->net = net;
    job->out.resize(1);
    TargetOut &o = job->out[0];
    Work w;
    int rc = alloc_work(w, net, lim, 0, s);
    unsigned long long h[C_COUNT];
    auto fail = [&](int code) {
        cudaGetLastError();
        free_work(w, s);
        efm_free_job(job);
        return code;
    };
    if (rc != EFM_OK) return fail(rc);
    LevelArgs a{};
    a.cslots = (unsigned long long *)w.cslots.p;
    a.cslot_mask = w.cslot_cap - 1;
    a.cand = (uint64_t *)w.cand.p;
    a.cand_cap = w.cand_cap;
    a.max_len = lim.max_len;
    a.max_sec = lim.max_secondary;
    a.ctr = (unsigned long long *)w.ctr.p;
    AcceptArgs acc{};
    acc.cand = (const uint64_t *)w.cand.p;
    acc.res = (uint64_t *)w.res.p;
    acc.res_cap = w.res_cap;
    acc.rcols = nv.W > 2 ? (uint16_t *)w.rcols.p : nullptr;
    acc.ctr = a.ctr;
    auto sync_ctr = [&]() -> int {
        if (cudaMemcpyAsync(h, a.ctr, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return EFM_ECUDA;
        return err_from_bits(h[C_ERR]);
    };
    float ms = 0.f;
    if (cudaMemsetAsync(a.ctr, 0, C_COUNT * 8, s) != cudaSuccess ||
        cudaMemsetAsync(w.cslots.p, 0xFF, w.cslot_cap * 8, s) != cudaSuccess || cudaEventRecord(w.ev[0], s) != cudaSuccess ||
        launch_walks(nv, a, target, seed, n_walks, net->sm_count, s) != cudaSuccess || cudaEventRecord(w.ev[2], s) != cudaSuccess)
        return fail(EFM_ECUDA);
    if ((rc = sync_ctr())) return fail(rc);
    acc.cand_begin = 0;
    acc.cand_end = (int64_t)h[C_CAND_N];
    if (launch_accept(nv, acc, s) != cudaSuccess) return fail(EFM_ECUDA);
    if ((rc = sync_ctr())) return fail(rc);
    if ((int64_t)h[C_RES_N] > w.res_cap) return fail(EFM_ECAPACITY);
    const int64_t res_n = (int64_t)h[C_RES_N];
    const uint64_t n2 = next_pow2((uint64_t)std::max<int64_t>(res_n, 1));
    if (!dev_alloc(w.sortidx, n2 * 4, s) || !dev_alloc(o.sup, (size_t)std::max<int64_t>(res_n, 1) * nv.W * 8, s))
        return fail(EFM_ENOMEM);
    if (launch_sort_results((const uint64_t *)w.res.p, res_n, nv.W, (uint32_t *)w.sortidx.p, (int64_t)n2,
                            (uint64_t *)o.sup.p, res_n, s) != cudaSuccess ||
        cudaEventRecord(w.ev[1], s) != cudaSuccess || cudaEventSynchronize(w.ev[1]) != cudaSuccess)
        return fail(EFM_ECUDA);
    cudaEventElapsedTime(&ms, w.ev[0], w.ev[1]);
    o.total_ms = ms;
    cudaEventElapsedTime(&ms, w.ev[0], w.ev[2]);
    o.expand_ms = ms;  // the walk kernel
    o.expand_launches = n_walks > 0 ? 1 : 0;
    o.kernel_launches = 2 + (res_n > 0 ? 2 : 0);
    o.n = res_n;
    efm_counters &c = o.ctr;
    memset(&c, 0, sizeof(c));
    c.levels = (int64_t)h[C_LEVELS];
    c.seeds = (int64_t)h[C_SEEDS];
    c.expansions = (int64_t)h[C_EXP];
    c.overflow = (int64_t)h[C_OVF];
    c.balanced = (int64_t)h[C_BAL];
    c.candidates = (int64_t)h[C_CAND_N];
    c.results = (int64_t)h[C_RES];
    c.pruned = (int64_t)h[C_PRUNED];
    c.status = c.overflow ? EFM_OVERFLOW_DROPPED : 0;
    o.status = (int)c.status;
    free_work(w, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        efm_free_job(job);
        return EFM_ECUDA;
    }
    *out = job;
    return o.status;
}

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Scratch slice of one CTA of the batched traversal, sized for the largest
// network of the batch.
BatchLayout batch_layout(int64_t cap, int Wmax, int Mpad_max, int Nmax, int max_len_max)
{
    BatchLayout L{};
    L.cap = cap;
    L.cand_cap = (int64_t)1 << 15;
    L.res_cap = (int64_t)1 << 13;
    L.slot_cap = next_pow2(2 * (uint64_t)cap + 64 * (uint64_t)(kBatchThreads / 32));
    L.cslot_cap = next_pow2(2 * (uint64_t)L.cand_cap);
    size_t o = 0;
    for (int i = 0; i < 2; ++i) {
        L.o_U[i] = o;
        o = align256(o + (size_t)cap * Wmax * 8);
        L.o_B[i] = o;
        o = align256(o + (size_t)cap * Mpad_max * 4);
        L.o_meta[i] = o;
        o = align256(o + (size_t)cap * 4);
    }
    L.o_slots = o;
    o = align256(o + L.slot_cap * 8);
    L.o_cslots = o;
    o = align256(o + L.cslot_cap * 8);
    L.o_cand = o;
    o = align256(o + (size_t)L.cand_cap * Wmax * 8);
    L.o_res = o;
    o = align256(o + (size_t)L.res_cap * Wmax * 8);
    L.o_bcnt = o;
    o = align256(o + (size_t)Nmax * 4);
    L.o_bfill = o;
    o = align256(o + (size_t)Nmax * 4);
    L.o_bptr = o;
    o = align256(o + (size_t)(Nmax + 1) * 4);
    L.o_bres = o;
    o = align256(o + (size_t)L.res_cap * max_len_max * Wmax * 8);
    L.o_sort = o;
    o = align256(o + next_pow2((uint64_t)L.res_cap) * 4);
    L.o_rcols = o;
    o = align256(o + (Wmax > 2 ? (size_t)L.res_cap * kRcolStride * 2 : 16));
    L.slice_bytes = o;
    return L;
}

// Autotuner: a launch configuration of the batched traversal, and its cache
// keyed by (log2 jobs, largest row class, SMs).  A pinned configuration
// (efm_batch_set_tuning) replaces the search.
struct TuneChoice {
    int per_sm = 1, big = 1, warps = 8, tile = 32, chunk = 1;
    float default_ms = 0.f, best_ms = 0.f;  // the sample's time: untuned and chosen configuration
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, TuneChoice> g_tune;
TuneChoice g_last;
bool g_have_last = false, g_pinned = false;
TuneChoice g_pin;

}  // namespace

extern "C" int efm_find_pathways_batch(efm_net *const *nets, const int32_t *targets, int32_t n_jobs,
                                       const efm_limits *limits, const efm_model *model, efm_job **out)
{
    if (!out) return EFM_EINVAL;
    *out = nullptr;
    if (!nets || !targets || n_jobs <= 0 || !limits || model) return EFM_EINVAL;
    const efm_limits lim = *limits;
    if (lim.max_len < 1 || lim.max_len > EFM_MAX_LEN || lim.max_secondary < 0 || lim.first_k != 0 ||
        lim.proposal != 0 || lim.max_frontier <= 0 || lim.variant != EFM_ADDITIVE || lim.reserved != 0)
        return EFM_EINVAL;
    int Wmax = 1, Mpad_max = 32, Nmax = 1, Lmax = 1, max_epl = 1;
    for (int i = 0; i < n_jobs; ++i) {
        const efm_net *n = nets[i];
        if (!n || targets[i] < -1 || targets[i] >= n->n_met) return EFM_EINVAL;
        if (n->nv.EPL > 8) return EFM_EUNSUPPORTED;
        Wmax = std::max(Wmax, n->nv.W);
        Mpad_max = std::max(Mpad_max, n->nv.Mpad);
        Nmax = std::max(Nmax, n->nv.N);
        Lmax = std::max(Lmax, std::min(lim.max_len, n->nv.N));
        max_epl = std::max(max_epl, n->nv.EPL);
    }
    efm_net *net0 = nets[0];
    cudaStream_t s = net0->stream;
    const BatchLayout L = batch_layout(lim.max_frontier + 1, Wmax, Mpad_max, Nmax, Lmax);
    const int occ8 = batch_blocks_per_sm(8), occ4 = batch_blocks_per_sm(4);
    const int occ = std::max(occ8, occ4);  // slices for the largest grid any configuration launches
    const int sms = net0->sm_count;

    auto *job = new (std::nothrow) efm_job();
    if (!job) return EFM_ENOMEM;
    job->net = net0;
    job->out.resize(n_jobs);
    job->words.resize(n_jobs);
    DevBuf pool, djobs, dorder, dctr, dqueue;
    const size_t out_rows = (size_t)L.res_cap;
    int rc = EFM_OK;
    std::vector<BatchJob> hj(n_jobs);
    std::vector<int> order_in(n_jobs), order_big(n_jobs);
    std::vector<unsigned long long> hctr((size_t)n_jobs * C_COUNT);
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    TuneChoice best;
    BatchArgs ba{};

    if (!dev_alloc(pool, (size_t)sms * occ * L.slice_bytes, s) ||
        !dev_alloc(djobs, sizeof(BatchJob) * (size_t)n_jobs, s) || !dev_alloc(dorder, 4 * (size_t)n_jobs, s) ||
        !dev_alloc(dctr, 8 * (size_t)C_COUNT * n_jobs, s) || !dev_alloc(dqueue, 16, s) ||
        !dev_alloc(job->shared_out, out_rows * Wmax * 8 * (size_t)n_jobs, s)) {
        rc = EFM_ENOMEM;
        goto done;
    }
    for (int i = 0; i < n_jobs; ++i) {
        hj[i].nv = nets[i]->nv;
        hj[i].target = targets[i];
        hj[i].max_len = std::min(lim.max_len, nets[i]->nv.N);
        hj[i].out = (uint64_t *)job->shared_out.p + (size_t)i * out_rows * Wmax;
        hj[i].ctr = (unsigned long long *)dctr.p + (size_t)i * C_COUNT;
        order_in[i] = i;
        order_big[i] = i;
        job->words[i] = nets[i]->nv.W;
    }
    // queue schedule "largest first": by the number of split columns times
    // internal metabolites (a proxy of the traversal's size)
    std::stable_sort(order_big.begin(), order_big.end(), [&](int x, int y) {
        return (int64_t)nets[x]->nv.N * nets[x]->nv.M > (int64_t)nets[y]->nv.N * nets[y]->nv.M;
    });
    if (cudaMemcpyAsync(djobs.p, hj.data(), sizeof(BatchJob) * n_jobs, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = EFM_ECUDA;
        goto done;
    }
    ba.jobs = (const BatchJob *)djobs.p;
    ba.order = (const int *)dorder.p;
    ba.queue = (unsigned int *)dqueue.p;
    ba.pool = (char *)pool.p;
    ba.layout = L;
    ba.max_sec = lim.max_secondary;
    ba.max_frontier = lim.max_frontier;
    ba.max_results = lim.max_results;
    {
        // autotune on a sample of the jobs, cached per shape: CTAs per SM and
        // the queue order, then warps per job, then the parents a warp takes
        // per pass, then the queue positions a CTA claims at a time
        int lg = 0;
        while ((1 << lg) < n_jobs) ++lg;
        const auto key = std::make_tuple(lg, max_epl, sms);
        bool have = false;
        {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            if (g_pinned) {
                best = g_pin;
                if (best.per_sm == 0) best.per_sm = best.warps == 8 ? occ8 : occ4;  // every CTA the SM holds
                have = true;
            } else {
                auto it = g_tune.find(key);
                if (it != g_tune.end()) {
                    best = it->second;
                    have = true;
                }
            }
        }
        if (!have && n_jobs >= 64) {
            const int sample = std::min(n_jobs, 256);
            auto time_cfg = [&](const TuneChoice &c, float &t) -> bool {
                const std::vector<int> &ord = c.big ? order_big : order_in;
                // a strided sample keeps the size mix of the whole batch
                std::vector<int> samp(sample);
                for (int i = 0; i < sample; ++i) samp[i] = ord[(size_t)i * n_jobs / sample];
                ba.n_jobs = sample;
                ba.tile = c.tile;
                ba.chunk = c.chunk;
                if (cudaMemcpyAsync(dorder.p, samp.data(), 4 * sample, cudaMemcpyHostToDevice, s) != cudaSuccess ||
                    cudaMemsetAsync(dctr.p, 0, 8 * (size_t)C_COUNT * n_jobs, s) != cudaSuccess ||
                    cudaMemsetAsync(dqueue.p, 0, 16, s) != cudaSuccess || cudaEventRecord(e0, s) != cudaSuccess ||
                    launch_batch(ba, sms * c.per_sm, c.warps, s) != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
                    cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
                    if (getenv("EFM_DEBUG"))
                        fprintf(stderr, "efm: batch tuning run failed: %s\n", cudaGetErrorString(cudaGetLastError()));
                    return false;
                }
                if (getenv("EFM_DEBUG"))
                    fprintf(stderr, "efm: tune per_sm %d big %d warps %d tile %d chunk %d: %.3f ms\n", c.per_sm, c.big,
                            c.warps, c.tile, c.chunk, t);
                return true;
            };
            // the untuned configuration: 8 warps, every CTA the SM holds, queue in input order
            TuneChoice cur;
            cur.per_sm = occ8;
            cur.big = 0;
            float t = 0.f, best_t = 0.f;
            bool ok = time_cfg(cur, t);
            best = cur;
            best_t = t;
            const float def_t = t;
            auto consider = [&](const TuneChoice &c) {
                if (ok && (ok = time_cfg(c, t)) && t < best_t) {
                    best = c;
                    best_t = t;
                }
            };
            for (int big = 0; big < 2; ++big)
                for (int per_sm = 1; per_sm <= occ8; ++per_sm) {
                    cur = best;
                    cur.big = big;
                    cur.per_sm = per_sm;
                    cur.warps = 8;
                    if (!(big == 0 && per_sm == occ8)) consider(cur);
                }
            for (int per_sm = 1; per_sm <= occ4; ++per_sm) {
                cur = best;
                cur.warps = 4;
                cur.per_sm = per_sm;
                consider(cur);
            }
            for (int tile : {8, 16}) {
                cur = best;
                cur.tile = tile;
                consider(cur);
            }
            for (int chunk : {2, 4}) {
                cur = best;
                cur.chunk = chunk;
                consider(cur);
            }
            if (!ok) {
                rc = EFM_ECUDA;
            } else {
                best.default_ms = def_t;
                best.best_ms = best_t;
                std::lock_guard<std::mutex> lock(g_tune_mu);
                g_tune[key] = best;
            }
        }
        if (rc == EFM_OK) {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            g_last = best;
            g_have_last = true;
        }
    }
    if (rc != EFM_OK) goto done;
    // the batch: one persistent launch, captured in a CUDA graph with its resets
    ba.n_jobs = n_jobs;
    ba.tile = best.tile;
    ba.chunk = best.chunk;
    if (cudaMemcpyAsync(dorder.p, (best.big ? order_big : order_in).data(), 4 * (size_t)n_jobs,
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        rc = EFM_ECUDA;
        goto done;
    }
    {
        // capture on a private stream (the caller's may be the legacy default
        // stream, which cannot be captured); the graph then runs on the caller's
        cudaStream_t cs = nullptr;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
            rc = EFM_ECUDA;
            goto done;
        }
        bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            ok = cudaMemsetAsync(dctr.p, 0, 8 * (size_t)C_COUNT * n_jobs, cs) == cudaSuccess &&
                 cudaMemsetAsync(dqueue.p, 0, 16, cs) == cudaSuccess &&
                 launch_batch(ba, sms * best.per_sm, best.warps, cs) == cudaSuccess;
            ok = (cudaStreamEndCapture(cs, &graph) == cudaSuccess) && ok;
        }
        ok = ok && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
        cudaStreamDestroy(cs);
        if (!ok) {
            if (getenv("EFM_DEBUG")) fprintf(stderr, "efm: batch graph capture failed: %s\n", cudaGetErrorString(cudaGetLastError()));
            rc = EFM_ECUDA;
            goto done;
        }
    }
    if (cudaEventRecord(e0, s) != cudaSuccess || cudaGraphLaunch(exec, s) != cudaSuccess ||
        cudaEventRecord(e1, s) != cudaSuccess ||
        cudaMemcpyAsync(hctr.data(), dctr.p, 8 * hctr.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        if (getenv("EFM_DEBUG")) fprintf(stderr, "efm: batch launch failed: %s\n", cudaGetErrorString(cudaGetLastError()));
        rc = EFM_ECUDA;
        goto done;
    }
    for (int i = 0; i < n_jobs; ++i) {
        const unsigned long long *h = &hctr[(size_t)i * C_COUNT];
        TargetOut &o = job->out[i];
        o.borrowed = hj[i].out;
        o.err = err_from_bits(h[C_ERR]);
        if (!o.err && !h[C_DONE]) o.err = EFM_ECUDA;
        o.n = (int64_t)h[C_OUT_N];
        efm_counters &c = o.ctr;
        c.levels = (int64_t)h[C_LEVELS];
        c.seeds = (int64_t)h[C_SEEDS];
        c.expansions = (int64_t)h[C_EXP];
        c.overflow = (int64_t)h[C_OVF];
        c.balanced = (int64_t)h[C_BAL];
        c.candidates = (int64_t)h[C_CAND_N];
        c.results = (int64_t)h[C_RES];
        c.pruned = (int64_t)h[C_PRUNED];
        c.frontier = (int64_t)h[C_FRONTIER];
        c.frontier_max = (int64_t)h[C_FRONTIER_MAX];
        c.status = (int64_t)h[C_STATUS];
        o.status = (int)h[C_STATUS];
        o.total_ms = ms;
        o.kernel_launches = i == 0 ? 1 : 0;
    }
done:
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(pool, s);
    dev_free(djobs, s);
    dev_free(dorder, s);
    dev_free(dctr, s);
    dev_free(dqueue, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == EFM_OK) rc = EFM_ECUDA;
    if (rc != EFM_OK) {
        cudaGetLastError();
        efm_free_job(job);
        return rc;
    }
    int flags = 0;
    for (auto &o : job->out) flags |= o.status;
    *out = job;
    return flags;
}

extern "C" int efm_batch_tuning(efm_batch_tune *out)
{
    if (!out) return EFM_EINVAL;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    if (!g_have_last) return EFM_EINVAL;
    const TuneChoice &v = g_last;
    out->ctas_per_sm = v.per_sm;
    out->largest_first = v.big;
    out->warps_per_job = v.warps;
    out->tile = v.tile;
    out->queue_chunk = v.chunk;
    out->pinned = g_pinned ? 1 : 0;
    out->sample_default_ms = v.default_ms;
    out->sample_tuned_ms = v.best_ms;
    return EFM_OK;
}

extern "C" int efm_batch_set_tuning(const efm_batch_tune *cfg)
{
    if (!cfg) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_pinned = false;
        return EFM_OK;
    }
    if ((cfg->warps_per_job != 4 && cfg->warps_per_job != 8) || cfg->largest_first < 0 || cfg->largest_first > 1 ||
        cfg->tile < 1 || cfg->tile > 32 || cfg->queue_chunk < 1 || cfg->queue_chunk > 64 || cfg->ctas_per_sm < 0)
        return EFM_EINVAL;
    if (cfg->ctas_per_sm > batch_blocks_per_sm(cfg->warps_per_job)) return EFM_EINVAL;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_pin = TuneChoice{};
    g_pin.per_sm = cfg->ctas_per_sm;
    g_pin.big = cfg->largest_first;
    g_pin.warps = cfg->warps_per_job;
    g_pin.tile = cfg->tile;
    g_pin.chunk = cfg->queue_chunk;
    g_pinned = true;
    return EFM_OK;
}

extern "C" int efm_fetch_results(efm_job *job, int32_t idx, uint64_t *supports, int64_t capacity, int64_t *n_out,
                                 int32_t *words_per_set, efm_counters *ctr)
{
    if (!job || idx < 0 || idx >= (int32_t)job->out.size()) return EFM_EINVAL;
    TargetOut &o = job->out[idx];
    const int W = job->words.empty() ? job->net->nv.W : job->words[idx];
    if (n_out) *n_out = o.n;
    if (words_per_set) *words_per_set = W;
    if (ctr) *ctr = o.ctr;
    if (o.err) return o.err;
    if (!supports) return o.status;
    if (capacity < o.n) return EFM_ECAPACITY;
    if (o.n > 0) {
        const void *src = o.borrowed ? (const void *)o.borrowed : o.sup.p;
        if (cudaMemcpyAsync(supports, src, (size_t)o.n * W * 8, cudaMemcpyDeviceToHost, job->net->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(job->net->stream) != cudaSuccess) {
            cudaGetLastError();
            return EFM_ECUDA;
        }
    }
    return o.status;
}

extern "C" int efm_job_timing(const efm_job *job, int32_t idx, double *total_ms, double *expand_ms,
                              int64_t *expand_launches, double *expand_bytes, int64_t *kernel_launches)
{
    if (!job || idx < 0 || idx >= (int32_t)job->out.size()) return EFM_EINVAL;
    const TargetOut &o = job->out[idx];
    if (total_ms) *total_ms = o.total_ms;
    if (expand_ms) *expand_ms = o.expand_ms;
    if (expand_launches) *expand_launches = o.expand_launches;
    if (expand_bytes) *expand_bytes = o.expand_bytes;
    if (kernel_launches) *kernel_launches = o.kernel_launches;
    return EFM_OK;
}

extern "C" void efm_free_job(efm_job *job)
{
    if (!job) return;
    cudaStream_t s = job->net ? job->net->stream : nullptr;
    for (auto &o : job->out) dev_free(o.sup, s);
    dev_free(job->shared_out, s);
    cudaStreamSynchronize(s);
    delete job;
}

// ---------------------------------------------------------------------------
// Proposal model (the learned order of first-K searches).
// ---------------------------------------------------------------------------

namespace {

uint64_t splitmix64(uint64_t &x)
{
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

float uniform_pm1(uint64_t &x) { return (float)((double)(splitmix64(x) >> 11) * (2.0 / 9007199254740992.0) - 1.0); }

int model_check_err(efm_model *m)
{
    unsigned e = 0;
    if (cudaMemcpyAsync(&e, m->err.p, 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess) {
        cudaGetLastError();
        return EFM_ECUDA;
    }
    return e ? EFM_ETIMEOUT : EFM_OK;
}

// valid rows in training tile t
int64_t tile_rows(const efm_model *m, int64_t t) { return std::min<int64_t>(kMlpTileRows, m->n_rows - t * kMlpTileRows); }

bool model_reserve_rows(efm_model *m, int64_t rows)
{
    const int64_t need = (rows + kMlpTileRows - 1) / kMlpTileRows * kMlpTileRows;
    if (need <= m->cap_rows) return true;
    const int64_t cap = std::max<int64_t>(need, 2 * m->cap_rows);
    DevBuf X, y, tiles;
    if (!dev_alloc(X, (size_t)cap * kMlpFeatures * 2, m->stream) || !dev_alloc(y, (size_t)cap * 4, m->stream) ||
        !dev_alloc(tiles, (size_t)(cap / kMlpTileRows) * 4, m->stream)) {
        dev_free(X, m->stream);
        dev_free(y, m->stream);
        dev_free(tiles, m->stream);
        return false;
    }
    // rows past n_rows stay zero (padding of the last tile)
    cudaMemsetAsync(X.p, 0, (size_t)cap * kMlpFeatures * 2, m->stream);
    if (m->n_rows > 0) {
        const int64_t used = (m->n_rows + kMlpTileRows - 1) / kMlpTileRows * kMlpTileRows;
        cudaMemcpyAsync(X.p, m->X.p, (size_t)used * kMlpFeatures * 2, cudaMemcpyDeviceToDevice, m->stream);
        cudaMemcpyAsync(y.p, m->y.p, (size_t)m->n_rows * 4, cudaMemcpyDeviceToDevice, m->stream);
    }
    dev_free(m->X, m->stream);
    dev_free(m->y, m->stream);
    dev_free(m->tiles, m->stream);
    // the rows may be written from another stream (a network's, when tracing)
    cudaStreamSynchronize(m->stream);
    m->X = X;
    m->y = y;
    m->tiles = tiles;
    m->cap_rows = cap;
    return true;
}

}  // namespace

extern "C" int efm_model_create(uint64_t seed, uintptr_t cuda_stream, efm_model **out)
{
    if (!out) return EFM_EINVAL;
    *out = nullptr;
    auto *m = new (std::nothrow) efm_model();
    if (!m) return EFM_ENOMEM;
    m->stream = (cudaStream_t)cuda_stream;
    cudaStream_t s = m->stream;
    const size_t pb = (size_t)kMlpParams * 4;
    if (!dev_alloc(m->params, pb, s) || !dev_alloc(m->grad, pb, s) || !dev_alloc(m->mom, 2 * pb, s) ||
        !dev_alloc(m->wb, (size_t)kMlpHidden * kMlpFeatures * 2, s) || !dev_alloc(m->loss, 4, s) ||
        !dev_alloc(m->err, 4, s)) {
        efm_model_free(m);
        return EFM_ENOMEM;
    }
    // uniform initialisation scaled by fan-in (He), from a seeded splitmix64 stream
    std::vector<float> p((size_t)kMlpParams, 0.f);
    uint64_t st = seed;
    const float a1 = std::sqrt(6.0f / kMlpFeatures), a2 = std::sqrt(3.0f / kMlpHidden);
    for (int i = 0; i < kMlpW2; ++i) p[kMlpW1 + i] = a1 * uniform_pm1(st);
    for (int j = 0; j < kMlpHidden; ++j) p[kMlpW2 + j] = a2 * uniform_pm1(st);
    p[kMlpB2] = 0.f;
    if (cudaMemcpyAsync(m->params.p, p.data(), pb, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(m->grad.p, 0, pb, s) != cudaSuccess || cudaMemsetAsync(m->mom.p, 0, 2 * pb, s) != cudaSuccess ||
        cudaMemsetAsync(m->err.p, 0, 4, s) != cudaSuccess ||
        launch_pack_w((const float *)m->params.p, m->wb.p, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        efm_model_free(m);
        return EFM_ECUDA;
    }
    *out = m;
    return EFM_OK;
}

extern "C" int efm_model_params(efm_model *m, float *params, int32_t write)
{
    if (!m || !params) return EFM_EINVAL;
    cudaStream_t s = m->stream;
    const size_t pb = (size_t)kMlpParams * 4;
    if (write) {
        if (cudaMemcpyAsync(m->params.p, params, pb, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemsetAsync(m->mom.p, 0, 2 * pb, s) != cudaSuccess ||
            launch_pack_w((const float *)m->params.p, m->wb.p, s) != cudaSuccess) {
            cudaGetLastError();
            return EFM_ECUDA;
        }
        m->step = 0;
    } else if (cudaMemcpyAsync(params, m->params.p, pb, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
        cudaGetLastError();
        return EFM_ECUDA;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return EFM_ECUDA;
    }
    return EFM_OK;
}

extern "C" int efm_model_add_rows(efm_model *m, const float *x, const float *y, int64_t n)
{
    if (!m || n < 0 || (n > 0 && (!x || !y))) return EFM_EINVAL;
    if (n == 0) return EFM_OK;
    for (int64_t i = 0; i < n; ++i)
        if (!(y[i] == 0.f || y[i] == 1.f)) return EFM_EINVAL;
    cudaStream_t s = m->stream;
    if (!model_reserve_rows(m, m->n_rows + n)) return EFM_ENOMEM;
    DevBuf tmp;
    if (!dev_alloc(tmp, (size_t)n * kMlpFeatures * 4, s)) return EFM_ENOMEM;
    int rc = EFM_OK;
    if (cudaMemcpyAsync(tmp.p, x, (size_t)n * kMlpFeatures * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        launch_pack_rows((const float *)tmp.p, n, m->X.p, m->n_rows, s) != cudaSuccess ||
        cudaMemcpyAsync((float *)m->y.p + m->n_rows, y, (size_t)n * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        rc = EFM_ECUDA;
    }
    dev_free(tmp, s);
    if (rc == EFM_OK) m->n_rows += n;
    return rc;
}

extern "C" int efm_model_rows(efm_model *m, int64_t *n_rows, int64_t *n_positive)
{
    if (!m) return EFM_EINVAL;
    if (n_rows) *n_rows = m->n_rows;
    if (n_positive) {
        std::vector<float> y((size_t)m->n_rows);
        if (m->n_rows > 0 &&
            (cudaMemcpyAsync(y.data(), m->y.p, y.size() * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
             cudaStreamSynchronize(m->stream) != cudaSuccess)) {
            cudaGetLastError();
            return EFM_ECUDA;
        }
        int64_t c = 0;
        for (float v : y) c += v > 0.5f;
        *n_positive = c;
    }
    return EFM_OK;
}

extern "C" int efm_model_clear_rows(efm_model *m)
{
    if (!m) return EFM_EINVAL;
    m->n_rows = 0;
    if (m->X.p && cudaMemsetAsync(m->X.p, 0, m->X.bytes, m->stream) != cudaSuccess) {
        cudaGetLastError();
        return EFM_ECUDA;
    }
    return EFM_OK;
}

extern "C" int efm_model_forward(efm_model *m, const float *x, int64_t n, float *scores)
{
    if (!m || n < 0 || (n > 0 && (!x || !scores))) return EFM_EINVAL;
    if (n == 0) return EFM_OK;
    cudaStream_t s = m->stream;
    const int64_t rows = (n + kMlpTileRows - 1) / kMlpTileRows * kMlpTileRows;
    DevBuf tx, tX, ts;
    int rc = EFM_OK;
    if (!dev_alloc(tx, (size_t)n * kMlpFeatures * 4, s) || !dev_alloc(tX, (size_t)rows * kMlpFeatures * 2, s) ||
        !dev_alloc(ts, (size_t)n * 4, s)) {
        rc = EFM_ENOMEM;
    } else if (cudaMemcpyAsync(tx.p, x, (size_t)n * kMlpFeatures * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
               cudaMemsetAsync(tX.p, 0, (size_t)rows * kMlpFeatures * 2, s) != cudaSuccess ||
               launch_pack_rows((const float *)tx.p, n, tX.p, 0, s) != cudaSuccess ||
               launch_mlp_score(tX.p, n, m->wb.p, (const float *)m->params.p, (float *)ts.p, (unsigned *)m->err.p,
                                s) != cudaSuccess ||
               cudaMemcpyAsync(scores, ts.p, (size_t)n * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
               cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        rc = EFM_ECUDA;
    }
    dev_free(tx, s);
    dev_free(tX, s);
    dev_free(ts, s);
    if (rc == EFM_OK) rc = model_check_err(m);
    return rc;
}

namespace {

// one training pass over tiles[0..n_tiles) (device list); adds the gradient
// into m->grad and the loss into m->loss
int model_pass(efm_model *m, const int32_t *tiles_dev, int n_tiles, int64_t rows, float pos_weight)
{
    if (launch_mlp_train(m->X.p, (const float *)m->y.p, m->n_rows, tiles_dev, n_tiles, m->wb.p,
                         (const float *)m->params.p, pos_weight, 1.0f / (float)std::max<int64_t>(rows, 1),
                         (float *)m->grad.p, (float *)m->loss.p, (unsigned *)m->err.p, m->stream) != cudaSuccess) {
        cudaGetLastError();
        return EFM_ECUDA;
    }
    return EFM_OK;
}

}  // namespace

extern "C" int efm_model_gradient(efm_model *m, float pos_weight, float *grad, float *loss)
{
    if (!m || !grad || m->n_rows <= 0) return EFM_EINVAL;
    cudaStream_t s = m->stream;
    const int n_tiles = (int)((m->n_rows + kMlpTileRows - 1) / kMlpTileRows);
    std::vector<int32_t> t((size_t)n_tiles);
    for (int i = 0; i < n_tiles; ++i) t[i] = i;
    const size_t pb = (size_t)kMlpParams * 4;
    if (cudaMemcpyAsync(m->tiles.p, t.data(), t.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(m->grad.p, 0, pb, s) != cudaSuccess || cudaMemsetAsync(m->loss.p, 0, 4, s) != cudaSuccess) {
        cudaGetLastError();
        return EFM_ECUDA;
    }
    int rc = model_pass(m, (const int32_t *)m->tiles.p, n_tiles, m->n_rows, pos_weight);
    if (rc) return rc;
    float l = 0.f;
    if (cudaMemcpyAsync(grad, m->grad.p, pb, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&l, m->loss.p, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemsetAsync(m->grad.p, 0, pb, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return EFM_ECUDA;
    }
    if (loss) *loss = l;
    return model_check_err(m);
}

extern "C" int efm_model_train(efm_model *m, int32_t epochs, int32_t batch_tiles, float lr, float pos_weight,
                               uint64_t seed, float *last_loss)
{
    if (!m || epochs < 0 || batch_tiles < 1 || !(lr > 0.f) || !(pos_weight > 0.f) || m->n_rows <= 0)
        return EFM_EINVAL;
    cudaStream_t s = m->stream;
    const int n_tiles = (int)((m->n_rows + kMlpTileRows - 1) / kMlpTileRows);
    std::vector<int32_t> order((size_t)n_tiles);
    uint64_t st = seed;
    float epoch_loss = 0.f;
    for (int e = 0; e < epochs; ++e) {
        for (int i = 0; i < n_tiles; ++i) order[i] = i;
        for (int i = n_tiles - 1; i > 0; --i) std::swap(order[i], order[splitmix64(st) % (uint64_t)(i + 1)]);
        if (cudaMemcpyAsync(m->tiles.p, order.data(), order.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemsetAsync(m->loss.p, 0, 4, s) != cudaSuccess) {
            cudaGetLastError();
            return EFM_ECUDA;
        }
        int batches = 0;
        for (int b0 = 0; b0 < n_tiles; b0 += batch_tiles) {
            const int nb = std::min(batch_tiles, n_tiles - b0);
            int64_t rows = 0;
            for (int i = 0; i < nb; ++i) rows += tile_rows(m, order[b0 + i]);
            int rc = model_pass(m, (const int32_t *)m->tiles.p + b0, nb, rows, pos_weight);
            if (rc) return rc;
            if (launch_adam((float *)m->params.p, (float *)m->grad.p, (float *)m->mom.p, lr, ++m->step, m->wb.p, s) !=
                cudaSuccess) {
                cudaGetLastError();
                return EFM_ECUDA;
            }
            ++batches;
        }
        float l = 0.f;
        if (cudaMemcpyAsync(&l, m->loss.p, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return EFM_ECUDA;
        }
        epoch_loss = l / (float)std::max(batches, 1);
    }
    if (last_loss) *last_loss = epoch_loss;
    return model_check_err(m);
}

extern "C" int efm_model_trace(efm_model *m, efm_net *net, const int32_t *targets, int32_t n_targets,
                               const efm_limits *limits, int64_t rows_per_level)
{
    if (!m || !net || !targets || n_targets <= 0 || !limits || rows_per_level < 1) return EFM_EINVAL;
    efm_limits lim = *limits;
    lim.proposal = EFM_PLAIN;
    if (lim.max_len < 1 || lim.max_len > EFM_MAX_LEN || lim.max_secondary < 0 || lim.first_k <= 0 ||
        lim.max_results != 0 || lim.variant != EFM_ADDITIVE || lim.reserved != 0)
        return EFM_EINVAL;
    for (int i = 0; i < n_targets; ++i)
        if (targets[i] < -1 || targets[i] >= net->n_met) return EFM_EINVAL;
    Work w;
    const int total_warps = generate_grid(net->nv, net->sm_count) * kExpandWarps;
    int rc = alloc_work(w, net, lim, total_warps, net->stream);
    for (int i = 0; rc == EFM_OK && i < n_targets; ++i) {
        TargetOut ans;
        int depth = lim.max_len;
        rc = run_first_k(net, w, lim, targets[i], ans, nullptr, &depth);  // the answer, then the traced rerun
        if (rc == EFM_OK && ans.n > 0 && !(ans.status & EFM_TRUNCATED)) {
            Trace tr;
            tr.m = m;
            tr.ans = (const uint64_t *)ans.sup.p;
            tr.n_ans = ans.n;
            tr.rows_per_level = rows_per_level;
            TargetOut again;
            efm_limits last = lim;  // the search the answer came from: its last deepening run
            last.max_len = depth;
            rc = run_target(net, w, last, targets[i], again, nullptr, &tr);
            dev_free(again.sup, net->stream);
        }
        dev_free(ans.sup, net->stream);
    }
    free_work(w, net->stream);
    if (cudaStreamSynchronize(net->stream) != cudaSuccess && rc == EFM_OK) rc = EFM_ECUDA;
    cudaGetLastError();
    return rc;
}

extern "C" void efm_model_free(efm_model *m)
{
    if (!m) return;
    cudaStream_t s = m->stream;
    DevBuf *bufs[] = {&m->params, &m->grad, &m->mom, &m->wb, &m->loss, &m->err, &m->X, &m->y, &m->tiles};
    for (DevBuf *b : bufs) dev_free(*b, s);
    cudaStreamSynchronize(s);
    delete m;
}
